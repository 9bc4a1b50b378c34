// MSD radix partitioning on the GPU: Algorithm 1 of Leyenda (Section 3.1),
// re-designed for one GB300.
//
//   k_extract_*   the (key, pointer) tuples of Section 3.2, plus the histogram
//                 of the first radix ("compute a histogram based on the
//                 current radix", Section 3.1) and the bits in which keys differ.
//   k_hist        histogram of each big bucket's current digit (levels >= 1).
//   k_classify    Algorithm 1's control: a bucket above the big-bucket
//                 threshold recurses with a multi-CTA pass on the next digit,
//                 smaller ones go to the small-bucket queue (finish tasks);
//                 a digit that is the same for the whole bucket is skipped.
//   k_pass        ParallelRadixSort on one digit for all big buckets at once:
//                 per-warp match/ballot ranks, decoupled look-back prefix sums
//                 across the tiles of a bucket, and a scatter staged through
//                 shared memory so that each digit's run is written
//                 contiguously (the "cache aware scattering" of Section 3.1).
//   k_finish      the small-bucket queue: one CTA per task sorts it in shared
//                 memory by MSD counting passes, with comparison ranking for
//                 tiny sub-buckets (SingleThreadRadixSort / ComparisonSort of
//                 Algorithm 1), and emits the final permutation -- or, for
//                 100-byte records, gathers the records themselves into
//                 place (the record scatter of Section 3.2, fused).
#define LEY_FILE_ID 1
#include "ley_kernels.h"
#include "ley_rec100.cuh"
#include "ley_tma.cuh"

namespace ley {

using ull = unsigned long long;

// ------------------------------------------------------------- helpers

// Programmatic dependent launch: the level kernels are launched so that the
// next one may be scheduled while this one runs; each first waits for its
// predecessor's completion and memory (a no-op when launched plainly), then
// lets its own successor be scheduled.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t bswap32(uint32_t v) { return __byte_perm(v, 0, 0x0123); }

// Key byte d of a tuple (d in 0..11).
__device__ __forceinline__ uint32_t digit_of(const uint4& t, int d) {
    uint32_t w = d < 4 ? t.y : (d < 8 ? t.x : t.z);
    return (w >> (24 - 8 * (d & 3))) & 0xFFu;
}

__device__ __forceinline__ ull key_hi(const uint4& t) { return ((ull)t.y << 32) | t.x; }

// Stable key order on tuples: key bytes as unsigned integers, then index.
__device__ __forceinline__ bool tup_less(const uint4& a, const uint4& b, uint32_t lo_mask) {
    ull ka = key_hi(a), kb = key_hi(b);
    if (ka != kb) return ka < kb;
    uint32_t la = a.z & lo_mask, lb = b.z & lo_mask;
    if (la != lb) return la < lb;
    return a.w < b.w;
}

// First digit >= d whose byte is non-zero in the difference mask, or ndig.
__device__ __forceinline__ int first_varying_digit(ull dhi, uint32_t dlo, int d, int ndig) {
    for (int k = d; k < ndig; k++) {
        uint32_t b = k < 8 ? (uint32_t)(dhi >> (56 - 8 * k)) & 0xFFu
                           : (dlo >> (24 - 8 * (k - 8))) & 0xFFu;
        if (b) return k;
    }
    return ndig;
}

__device__ __forceinline__ ull ld_relaxed(const ull* p) {
    ull v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(ull* p, ull v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t sel8(const uint32_t (&w)[8], uint32_t q) {
    uint32_t v = w[0];
#pragma unroll
    for (int k = 1; k < 8; k++) v = (q == (uint32_t)k) ? w[k] : v;
    return v;
}

// Key of record i as a tuple (w = 0).  16-byte aligned vector loads of the
// one or two 16-byte chunks that hold the key bytes; a chunk is loaded only
// when it holds key bytes, so no load leaves the input buffer's 16-byte
// granules.
template <int REC>
__device__ __forceinline__ uint4 load_record_key(const uint8_t* __restrict__ in, ull i,
                                                 uint32_t rec_rt, uint32_t kb, const KeySpec& ks,
                                                 uint32_t koff = 0) {
    const uint32_t rec = REC ? (uint32_t)REC : rec_rt;
    ull s = i * rec + koff;  // the key (window) starts koff bytes into the record
    const uint4* p = reinterpret_cast<const uint4*>(in + (s & ~15ull));
    uint32_t o = (uint32_t)(s & 15);
    uint4 c0 = __ldg(p);
    uint4 c1 = make_uint4(0, 0, 0, 0);
    if (o + kb > 16) c1 = __ldg(p + 1);
    uint32_t w[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    uint32_t q = o >> 2, r = (o & 3) * 8;
    uint32_t a0 = sel8(w, q), a1 = sel8(w, q + 1), a2 = sel8(w, q + 2), a3 = sel8(w, q + 3);
    uint32_t u0 = __funnelshift_r(a0, a1, r);
    uint32_t u1 = __funnelshift_r(a1, a2, r);
    uint32_t u2 = __funnelshift_r(a2, a3, r);
    ull hi = (((ull)bswap32(u0) << 32) | bswap32(u1)) & ks.hi_mask;
    uint32_t lo = bswap32(u2) & ks.lo_mask;
    return make_uint4((uint32_t)hi, (uint32_t)(hi >> 32), lo, 0u);
}

// Block-wide OR of a (hi, lo) difference mask into shared words, then into
// the segment's global Diff.
__device__ __forceinline__ void warp_or_diff(ull dhi, uint32_t dlo, uint32_t* sh3) {
    uint32_t a = __reduce_or_sync(0xffffffffu, (uint32_t)(dhi >> 32));
    uint32_t b = __reduce_or_sync(0xffffffffu, (uint32_t)dhi);
    uint32_t c = __reduce_or_sync(0xffffffffu, dlo);
    if ((threadIdx.x & 31) == 0) {
        if (a) atomicOr(&sh3[0], a);
        if (b) atomicOr(&sh3[1], b);
        if (c) atomicOr(&sh3[2], c);
    }
}

__device__ __forceinline__ void flush_diff(const uint32_t* sh3, Diff* g) {
    ull hi = ((ull)sh3[0] << 32) | sh3[1];
    if (hi) atomicOr(&g->hi, hi);
    if (sh3[2]) atomicOr(&g->lo, sh3[2]);
}

// Histogram update with warp-level ballot aggregation: the lanes whose digit
// equals lane 0's add their count in one shared-memory atomic, the others
// add one each (digit 256 = no item).
__device__ __forceinline__ void hist_add_vote(uint32_t* sh_hist, uint32_t dg) {
    const uint32_t first = __shfl_sync(0xffffffffu, dg, 0);
    const uint32_t same = __ballot_sync(0xffffffffu, dg == first);
    if (dg == first) {
        if ((threadIdx.x & 31) == 0 && dg < 256u) atomicAdd(&sh_hist[dg], (uint32_t)__popc(same));
    } else if (dg < 256u) {
        atomicAdd(&sh_hist[dg], 1u);
    }
}

// Lanes of the warp whose 8-bit digit equals this lane's (multi-split by
// eight ballots, one per digit bit).
__device__ __forceinline__ uint32_t peers8(uint32_t dg) {
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; b++) {
        const bool bit = (dg >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bal : ~bal;
    }
    return m;
}

// Stable rank of this lane's item among the warp's items with the same digit
// so far: counter value before this step (returned by the group leader's
// shared-memory atomic, broadcast by shuffle) plus the lower lanes of the
// group.  The leaders of successive calls are different lanes, so the
// __syncwarp orders each call's atomics before the next call's.
__device__ __forceinline__ uint32_t warp_rank(uint32_t* cnt, uint32_t dg, bool valid,
                                              uint32_t lt_mask, int lane) {
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    const uint32_t peers = peers8(dg) & vmask;
    const int leader = valid ? __ffs(peers) - 1 : lane;
    uint32_t old = 0;
    if (valid && lane == leader) old = atomicAdd(&cnt[dg], (uint32_t)__popc(peers));
    __syncwarp();
    old = __shfl_sync(0xffffffffu, old, leader);
    return old + __popc(peers & lt_mask);
}

// The same rank without the atomic and the shuffle: every lane reads its
// digit's count (peers read the same word); then the lowest lane of each
// digit -- distinct digits of the warp's own row -- stores the count advanced
// by its peers.  Faster where few warps rank at once (the finishing CTAs);
// the atomic form is faster in the scatter pass.
// MATCH: the peers from one match instruction instead of the eight ballots
// (measured on the finishing kernel: faster for records, chiefly on skewed
// keys, slower for the 8-byte keys of pairs).
template <bool MATCH>
__device__ __forceinline__ uint32_t warp_rank_rw(uint32_t* cnt, uint32_t dg, bool valid,
                                                 uint32_t lt_mask) {
    uint32_t peers;
    if constexpr (MATCH) {
        peers = __match_any_sync(0xffffffffu, valid ? dg : 256u + (threadIdx.x & 31u));
    } else {
        const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
        peers = peers8(dg) & vmask;
    }
    const uint32_t old = valid ? cnt[dg] : 0u;
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) cnt[dg] = old + (uint32_t)__popc(peers);
    __syncwarp();
    return old + __popc(peers & lt_mask);
}

// ------------------------------------------------------------- extract

// One tile = kPassTile consecutive records: its digit counts go to
// tile_cnt[t] (the per-tile histogram of Section 3.1's "compute a histogram
// based on the current radix"), its tuples to tup in input order.
template <int REC>
__global__ void __launch_bounds__(256)
k_extract_records(const uint8_t* __restrict__ in, ull n, uint32_t rec_rt, KeySpec ks, Work w,
                  int hist_digit, uint32_t t_begin, uint32_t t_end, const uint8_t* ref_in) {
    __shared__ uint32_t sh_hist[kRadix];
    __shared__ uint32_t sh_d[3];
    if (threadIdx.x < 3) sh_d[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t kb = (uint32_t)ks.ndig;
    // The difference mask is taken against one fixed key (record 0 of the
    // whole input) in every launch over the input's tiles.
    const uint4 ref = load_record_key<REC>(ref_in, 0, rec_rt, kb, ks);
    uint4* __restrict__ tup = w.tup[0];
    ull dhi = 0;
    uint32_t dlo = 0;
    constexpr int U = 4;
    for (uint32_t t = t_begin + blockIdx.x; t < t_end; t += gridDim.x) {
        __syncthreads();
        sh_hist[threadIdx.x] = 0;
        __syncthreads();
        const ull base = (ull)t * kPassTile;
#pragma unroll 1
        for (int k0 = 0; k0 < kPassTile / 256; k0 += U) {
            uint4 tv[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const ull i = base + (k0 + u) * 256 + threadIdx.x;
                tv[u] = i < n ? load_record_key<REC>(in, i, rec_rt, kb, ks) : ref;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const ull i = base + (k0 + u) * 256 + threadIdx.x;
                uint32_t dg = 256u;
                if (i < n) {
                    tv[u].w = (uint32_t)i;
                    tup[i] = tv[u];
                    dg = digit_of(tv[u], hist_digit);
                    dhi |= key_hi(tv[u]) ^ key_hi(ref);
                    dlo |= tv[u].z ^ ref.z;
                }
                hist_add_vote(sh_hist, dg);
            }
        }
        __syncthreads();
        w.tile_cnt[(ull)t * kRadix + threadIdx.x] = sh_hist[threadIdx.x];
        if (threadIdx.x == 0) w.seg_tile_owner[0][t] = 0;
    }
    warp_or_diff(dhi, dlo, sh_d);
    __syncthreads();
    if (threadIdx.x == 0) flush_diff(sh_d, w.diff[0]);
}

// Keys longer than 12 bytes are sorted window by window, least significant
// 12-byte window first (LSD over windows, each window sorted by the MSD
// machinery): tuple j holds window [koff, koff + 12) of record order[j] --
// the order produced by the windows after this one (identity for the last
// window) -- and carries j, so that equal windows keep that order.
__global__ void __launch_bounds__(256)
k_extract_window(const uint8_t* __restrict__ in, const uint32_t* __restrict__ order, ull n,
                 uint32_t rec, uint32_t koff, KeySpec ks, Work w, uint32_t* err) {
    __shared__ uint32_t sh_hist[kRadix];
    __shared__ uint32_t sh_d[3];
    if (threadIdx.x < 3) sh_d[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t kb = (uint32_t)ks.ndig;
    const uint32_t r0 = order ? order[0] : 0u;
    const uint4 ref = load_record_key<0>(in, r0 < n ? r0 : 0, rec, kb, ks, koff);
    uint4* __restrict__ tup = w.tup[0];
    ull dhi = 0;
    uint32_t dlo = 0;
    const uint32_t ntiles = ceil_div_u64(n, kPassTile);
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();
        sh_hist[threadIdx.x] = 0;
        __syncthreads();
        const ull base = (ull)t * kPassTile;
#pragma unroll 1
        for (int k = 0; k < kPassTile / 256; k++) {
            const ull i = base + k * 256 + threadIdx.x;
            uint32_t dg = 256u;
            if (i < n) {
                uint32_t r = order ? order[i] : (uint32_t)i;
                if (r >= n) {  // never for a valid order; keeps reads in bounds
                    LEY_FAIL(err, kErrCapacity);
                    r = 0;
                }
                uint4 tv = load_record_key<0>(in, r, rec, kb, ks, koff);
                tv.w = (uint32_t)i;
                tup[i] = tv;
                dg = digit_of(tv, 0);
                dhi |= key_hi(tv) ^ key_hi(ref);
                dlo |= tv.z ^ ref.z;
            }
            hist_add_vote(sh_hist, dg);
        }
        __syncthreads();
        w.tile_cnt[(ull)t * kRadix + threadIdx.x] = sh_hist[threadIdx.x];
        if (threadIdx.x == 0) w.seg_tile_owner[0][t] = 0;
    }
    warp_or_diff(dhi, dlo, sh_d);
    __syncthreads();
    if (threadIdx.x == 0) flush_diff(sh_d, w.diff[0]);
}

// next[j] = order ? order[pass[j]] : pass[j]: the order after one more window.
__global__ void k_compose_order(const uint32_t* __restrict__ order, const uint32_t* __restrict__ pass,
                                uint32_t* __restrict__ next, ull n, uint32_t* err) {
    for (ull j = (ull)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (ull)gridDim.x * blockDim.x) {
        uint32_t p = pass[j];
        if (p >= n) {
            LEY_FAIL(err, kErrCapacity);
            p = 0;
        }
        next[j] = order ? order[p] : p;
    }
}

__global__ void __launch_bounds__(256)
k_extract_pairs(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ idx, ull n,
                Work w) {
    __shared__ uint32_t sh_hist[kRadix];
    __shared__ uint32_t sh_d[3];
    if (threadIdx.x < 3) sh_d[threadIdx.x] = 0;
    __syncthreads();
    const ull ref = __ldg(keys);
    uint4* __restrict__ tup = w.tup[0];
    ull dhi = 0;
    constexpr int U = 8;
    const uint32_t ntiles = ceil_div_u64(n, kPassTile);
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();
        sh_hist[threadIdx.x] = 0;
        __syncthreads();
        const ull base = (ull)t * kPassTile;
#pragma unroll 1
        for (int k0 = 0; k0 < kPassTile / 256; k0 += U) {
            ull kk[U];
            uint32_t vv[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const ull i = base + (k0 + u) * 256 + threadIdx.x;
                kk[u] = i < n ? __ldg(keys + i) : ref;
                vv[u] = i < n ? __ldg(idx + i) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const ull i = base + (k0 + u) * 256 + threadIdx.x;
                uint32_t dg = 256u;
                if (i < n) {
                    tup[i] = make_uint4((uint32_t)kk[u], (uint32_t)(kk[u] >> 32), vv[u], (uint32_t)i);
                    dg = (uint32_t)(kk[u] >> 56);
                    dhi |= kk[u] ^ ref;
                }
                hist_add_vote(sh_hist, dg);
            }
        }
        __syncthreads();
        w.tile_cnt[(ull)t * kRadix + threadIdx.x] = sh_hist[threadIdx.x];
        if (threadIdx.x == 0) w.seg_tile_owner[0][t] = 0;
    }
    warp_or_diff(dhi, 0u, sh_d);
    __syncthreads();
    if (threadIdx.x == 0) flush_diff(sh_d, w.diff[0]);
}

// ------------------------------------------------------------ batches
//
// A batch of R requests is one sort over R top-level segments: request r's
// tuples occupy [off_r, off_r + n_r) (off_r on a tile boundary), and the
// levels, the classification and the finish treat the requests as the
// buckets of a level -- an MSD pass never moves a tuple out of its bucket,
// so each request is sorted on its own, exactly as a single sort would.

// Level-0 segment list: one segment per request, its tiles, its zeroed
// key-difference mask.
__global__ void k_batch_setup(const BatchReq* __restrict__ reqs, uint32_t R, Work w,
                              uint32_t ntiles, int digit0) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        const BatchReq q = reqs[r];
        Seg s;
        s.start = q.off;
        s.count = (uint32_t)q.n;
        s.digit = (uint16_t)digit0;
        s.buf = 0;
        s.pad = 0;
        w.segs[0][r] = s;
        w.seg_tile_base[0][r] = (uint32_t)(q.off / kPassTile);
        Diff z;
        z.hi = 0;
        z.lo = 0;
        z.pad = 0;
        w.diff[0][r] = z;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        w.ctl->lvl[0].big_packed = ((ull)R << kPackShift) | ntiles;
}

// tile -> request (the last request starting at or before the tile), also
// the level-0 tile owners.
__global__ void k_batch_tiles(const BatchReq* __restrict__ reqs, uint32_t R, Work w,
                              uint32_t* __restrict__ tile_req, uint32_t ntiles) {
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles;
         t += gridDim.x * blockDim.x) {
        const ull pos = (ull)t * kPassTile;
        uint32_t lo = 0, hi = R;  // first request with off > pos
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (reqs[mid].off <= pos) lo = mid + 1;
            else hi = mid;
        }
        const uint32_t r = lo > 0 ? lo - 1 : 0;
        tile_req[t] = r;
        w.seg_tile_owner[0][t] = r;
    }
}

// Batch extract: tile t belongs to request tile_req[t]; its tuples carry
// indices local to the request; per-tile digit-0 counts as for one sort,
// and the difference mask against the request's first key goes to its
// segment.
template <int REC>
__global__ void __launch_bounds__(256)
k_batch_extract_records(const BatchReq* __restrict__ reqs, const uint32_t* __restrict__ tile_req,
                        uint32_t ntiles, uint32_t rec_rt, KeySpec ks, Work w, int hist_digit) {
    __shared__ uint32_t sh_hist[kRadix];
    __shared__ uint32_t sh_d[3];
    const uint32_t kb = (uint32_t)ks.ndig;
    uint4* __restrict__ tup = w.tup[0];
    constexpr int U = 4;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t r = tile_req[t];
        const BatchReq q = reqs[r];
        const uint8_t* in = q.in;
        const uint4 ref = load_record_key<REC>(in, 0, rec_rt, kb, ks);
        __syncthreads();
        sh_hist[threadIdx.x] = 0;
        if (threadIdx.x < 3) sh_d[threadIdx.x] = 0;
        __syncthreads();
        const ull lbase = (ull)t * kPassTile - q.off;  // first local index of the tile
        ull dhi = 0;
        uint32_t dlo = 0;
#pragma unroll 1
        for (int k0 = 0; k0 < kPassTile / 256; k0 += U) {
            uint4 tv[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const ull i = lbase + (k0 + u) * 256 + threadIdx.x;
                tv[u] = i < q.n ? load_record_key<REC>(in, i, rec_rt, kb, ks) : ref;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const ull i = lbase + (k0 + u) * 256 + threadIdx.x;
                uint32_t dg = 256u;
                if (i < q.n) {
                    tv[u].w = (uint32_t)i;
                    tup[q.off + i] = tv[u];
                    dg = digit_of(tv[u], hist_digit);
                    dhi |= key_hi(tv[u]) ^ key_hi(ref);
                    dlo |= tv[u].z ^ ref.z;
                }
                hist_add_vote(sh_hist, dg);
            }
        }
        warp_or_diff(dhi, dlo, sh_d);
        __syncthreads();
        w.tile_cnt[(ull)t * kRadix + threadIdx.x] = sh_hist[threadIdx.x];
        if (threadIdx.x == 0) flush_diff(sh_d, &w.diff[0][r]);
    }
}

__global__ void __launch_bounds__(256)
k_batch_extract_pairs(const BatchReq* __restrict__ reqs, const uint32_t* __restrict__ tile_req,
                      uint32_t ntiles, Work w) {
    __shared__ uint32_t sh_hist[kRadix];
    __shared__ uint32_t sh_d[3];
    uint4* __restrict__ tup = w.tup[0];
    constexpr int U = 8;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t r = tile_req[t];
        const BatchReq q = reqs[r];
        const uint64_t* keys = reinterpret_cast<const uint64_t*>(q.in);
        const ull ref = __ldg(keys);
        __syncthreads();
        sh_hist[threadIdx.x] = 0;
        if (threadIdx.x < 3) sh_d[threadIdx.x] = 0;
        __syncthreads();
        const ull lbase = (ull)t * kPassTile - q.off;
        ull dhi = 0;
#pragma unroll 1
        for (int k0 = 0; k0 < kPassTile / 256; k0 += U) {
            ull kk[U];
            uint32_t vv[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const ull i = lbase + (k0 + u) * 256 + threadIdx.x;
                kk[u] = i < q.n ? __ldg(keys + i) : ref;
                vv[u] = i < q.n ? __ldg(q.idx_in + i) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const ull i = lbase + (k0 + u) * 256 + threadIdx.x;
                uint32_t dg = 256u;
                if (i < q.n) {
                    tup[q.off + i] =
                        make_uint4((uint32_t)kk[u], (uint32_t)(kk[u] >> 32), vv[u], (uint32_t)i);
                    dg = (uint32_t)(kk[u] >> 56);
                    dhi |= kk[u] ^ ref;
                }
                hist_add_vote(sh_hist, dg);
            }
        }
        warp_or_diff(dhi, 0u, sh_d);
        __syncthreads();
        w.tile_cnt[(ull)t * kRadix + threadIdx.x] = sh_hist[threadIdx.x];
        if (threadIdx.x == 0) flush_diff(sh_d, &w.diff[0][r]);
    }
}

// Records of any size: out_r[j] = in_r[perm[off_r + j]], one warp per record
// (in words when the size is a multiple of 4, else in bytes).
__global__ void __launch_bounds__(256)
k_batch_gather_generic(const BatchReq* __restrict__ reqs, const uint32_t* __restrict__ tile_req,
                       const uint32_t* __restrict__ perm, ull npos, uint32_t rec, uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const ull warps = (ull)gridDim.x * (blockDim.x >> 5);
    const uint32_t words = rec / 4;
    for (ull pos = (ull)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pos < npos;
         pos += warps) {
        const BatchReq q = reqs[tile_req[pos / kPassTile]];
        if (pos - q.off >= q.n) continue;  // padding after the request's last tuple
        uint32_t pj = perm[pos];
        if (pj >= q.n) {  // never for a valid permutation; keeps reads in bounds
            if (lane == 0) LEY_FAIL(err, kErrCapacity);
            pj = 0;
        }
        if ((rec & 3u) == 0) {
            const uint32_t* sp = reinterpret_cast<const uint32_t*>(q.in + (ull)pj * rec);
            uint32_t* dp = reinterpret_cast<uint32_t*>(q.out + (pos - q.off) * rec);
            for (uint32_t k = lane; k < words; k += 32) dp[k] = __ldg(sp + k);
        } else {  // record sizes that are not a multiple of 4: bytes
            const uint8_t* sp = q.in + (ull)pj * rec;
            uint8_t* dp = q.out + (pos - q.off) * rec;
            for (uint32_t k = lane; k < rec; k += 32) dp[k] = __ldg(sp + k);
        }
    }
}

__global__ void k_init(Work w, ull n, int digit0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        w.ctl->lvl[0].big_packed = (1ull << kPackShift) | ceil_div_u64(n, kPassTile);
        Seg s;
        s.start = 0;
        s.count = (uint32_t)n;
        s.digit = (uint16_t)digit0;
        s.buf = 0;
        s.pad = 0;
        w.segs[0][0] = s;
        w.seg_tile_base[0][0] = 0;
    }
}

// ------------------------------------------------------------ histogram

// Per-tile digit counts of every big bucket of level L >= 1 (the tiles of a
// bucket are consecutive), and the bits in which each bucket's keys differ.
__global__ void __launch_bounds__(kHistThreads)
k_hist(Work w, KeySpec ks, int L) {
    __shared__ uint32_t sh_hist[kRadix];
    __shared__ uint32_t sh_d[3];
    pdl_enter();
    const int p = L & 1;
    const ull packed = w.ctl->lvl[L].big_packed;
    const uint32_t nseg = (uint32_t)(packed >> kPackShift);
    const uint32_t ntiles = (uint32_t)(packed & kPackMask);
    const int tid = threadIdx.x;
    if (nseg > w.cap_seg || ntiles > w.cap_tiles) {  // an append overflowed
        if (tid == 0 && blockIdx.x == 0) LEY_FAIL(w.err, kErrCapacity);
        return;
    }
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        __syncthreads();
        if (tid < kRadix) sh_hist[tid] = 0;
        if (tid < 3) sh_d[tid] = 0;
        // Thread 0 asks the L2 for this CTA's next tile (looked up in steps,
        // so that no load is waited for at once).
        const uint32_t tn = t + gridDim.x;
        uint32_t sn = kNoPass;
        if (tid == 0 && tn < ntiles) sn = w.seg_tile_owner[p][tn];
        __syncthreads();
        const uint32_t s = w.seg_tile_owner[p][t];
        const Seg sg = w.segs[p][s];
        if (s >= nseg || sg.start + sg.count > w.n || t < w.seg_tile_base[p][s] || sg.buf > 1) {
            if (tid == 0) LEY_FAIL(w.err, kErrCapacity);  // never for a valid list
            continue;
        }
        const uint32_t lt = t - w.seg_tile_base[p][s];
        const ull base = sg.start + (ull)lt * kPassTile;
        const uint32_t m = min((uint32_t)kPassTile, sg.count - lt * (uint32_t)kPassTile);
        const uint4* src = w.tup[sg.buf];
        const uint4 ref = src[sg.start];
        uint4 v[kHistItems];
#pragma unroll
        for (int k = 0; k < kHistItems; k++) {
            uint32_t idx = k * kHistThreads + tid;
            v[k] = idx < m ? src[base + idx] : ref;
        }
        Seg sgn;
        uint32_t tbn = 0;
        if (tid == 0 && sn < nseg) {
            sgn = w.segs[p][sn];
            tbn = w.seg_tile_base[p][sn];
        }
        ull dhi = 0;
        uint32_t dlo = 0;
#pragma unroll
        for (int k = 0; k < kHistItems; k++) {
            uint32_t idx = k * kHistThreads + tid;
            dhi |= key_hi(v[k]) ^ key_hi(ref);
            dlo |= v[k].z ^ ref.z;
            hist_add_vote(sh_hist, idx < m ? digit_of(v[k], sg.digit) : 256u);
        }
        warp_or_diff(dhi & ks.hi_mask, dlo & ks.lo_mask, sh_d);
        if (tid == 0 && sn < nseg && tn >= tbn && sgn.buf <= 1 && sgn.start + sgn.count <= w.n) {
            const ull off = (ull)(tn - tbn) * kPassTile;
            if (off < sgn.count) {
                const uint32_t mn = (uint32_t)min((ull)kPassTile, sgn.count - off);
                l2_prefetch_bulk(w.tup[sgn.buf] + sgn.start + off, mn * (uint32_t)sizeof(uint4));
            }
        }
        __syncthreads();
        if (tid < kRadix) w.tile_cnt[(ull)t * kRadix + tid] = sh_hist[tid];
        if (tid == 0) flush_diff(sh_d, &w.diff[p][s]);
    }
}

// ----------------------------------------------------------------- scan

constexpr ull kFlagAgg = 1ull << 62;
constexpr ull kFlagInc = 2ull << 62;
constexpr ull kValMask = (1ull << 56) - 1;

__device__ __forceinline__ ull pack_status(ull flag, int epoch, ull val) {
    return flag | ((ull)epoch << 56) | (val & kValMask);
}

// Turns the per-tile digit counts of level L into per-tile exclusive offsets
// inside each bucket (in place), and writes each bucket's total per digit.
// A single-pass segmented scan over chunks of kScanChunk tiles with
// decoupled look-back (Merrill & Garland): a chunk that contains the first
// tile of a bucket publishes its inclusive value at once; others publish
// their aggregate and sum predecessors' values until an inclusive one.
// Chunks are taken in order from a counter, so every predecessor of a chunk
// is already running.
__global__ void __launch_bounds__(kRadix)
k_scan(Work w, int L) {
    __shared__ uint32_t sh_own[kScanChunk];
    __shared__ uint8_t sh_head[kScanChunk];
    __shared__ uint8_t sh_last[kScanChunk];
    __shared__ uint32_t sh_chunk;
    pdl_enter();
    const int p = L & 1;
    const ull packed = w.ctl->lvl[L].big_packed;
    const uint32_t nseg = (uint32_t)(packed >> kPackShift);
    const uint32_t ntiles = (uint32_t)(packed & kPackMask);
    const uint32_t nchunks = ceil_div_u64(ntiles, kScanChunk);
    const int d = threadIdx.x;
    const int epoch = L + 1;
    if (nseg > w.cap_seg || ntiles > w.cap_tiles || nchunks > w.cap_chunks) {
        if (d == 0 && blockIdx.x == 0) LEY_FAIL(w.err, kErrCapacity);
        return;
    }
    while (true) {
        __syncthreads();
        if (d == 0) sh_chunk = atomicAdd(&w.ctl->lvl[L].scan_chunk_ctr, 1u);
        __syncthreads();
        const uint32_t k = sh_chunk;
        if (k >= nchunks) break;
        const uint32_t t0 = k * kScanChunk;
        const uint32_t nt = min((uint32_t)kScanChunk, ntiles - t0);
        if (d < (int)nt) {
            const uint32_t t = t0 + d;
            const uint32_t s = w.seg_tile_owner[p][t];
            sh_own[d] = s;
            sh_head[d] = s < nseg && w.seg_tile_base[p][s] == t;
            sh_last[d] = t + 1 == ntiles || w.seg_tile_owner[p][t + 1] != s;
        }
        __syncthreads();
        uint32_t c[kScanChunk], off[kScanChunk];
#pragma unroll
        for (int i = 0; i < kScanChunk; i++)
            c[i] = i < (int)nt ? w.tile_cnt[(ull)(t0 + i) * kRadix + d] : 0u;
        uint32_t run = 0;
        int first_head = (int)nt;
#pragma unroll
        for (int i = 0; i < kScanChunk; i++) {
            if (i < (int)nt && sh_head[i]) {
                run = 0;
                if (first_head == (int)nt) first_head = i;
            }
            off[i] = run;
            run += c[i];
        }
        ull* my = w.status + (ull)k * kRadix + d;
        const bool has_head = first_head < (int)nt;
        st_relaxed(my, pack_status(has_head ? kFlagInc : kFlagAgg, epoch, run));
        ull carry = 0;
        if (first_head > 0) {
            // Tiles before the chunk's first bucket start continue a bucket
            // from earlier chunks: look back for its running count.
            uint32_t j = k - 1;
            uint32_t spins = 0;
            while (true) {
                const ull sv = ld_relaxed(w.status + (ull)j * kRadix + d);
                const int ep = (int)((sv >> 56) & 0x3F);
                const ull flag = sv & (3ull << 62);
                if (ep != epoch || flag == 0) {
                    if (++spins > kSpinLimit) {
                        LEY_FAIL(w.err, kErrTimeout);
                        break;
                    }
                    if (spins > 32) __nanosleep(64);
                    continue;
                }
                carry += sv & kValMask;
                if (flag == kFlagInc || j == 0) break;
                j--;
            }
            if (!has_head) st_relaxed(my, pack_status(kFlagInc, epoch, carry + run));
        }
#pragma unroll
        for (int i = 0; i < kScanChunk; i++) {
            if (i < (int)nt) {
                const uint32_t o = off[i] + (i < first_head ? (uint32_t)carry : 0u);
                w.tile_cnt[(ull)(t0 + i) * kRadix + d] = o;
                if (sh_last[i] && sh_own[i] < nseg)
                    w.hist[p][(ull)sh_own[i] * kRadix + d] = o + c[i];
            }
        }
    }
}

// ------------------------------------------------------------- classify

// A finishing task.  A run whose keys are all equal (flags 1) is already in
// order and may be of any size; it is cut into pieces of at most kFlagPiece
// so that its output is written by many CTAs at once.
__device__ void emit_fin(const Work& w, ull start, uint32_t count, int digit, int buf, int flags) {
    const uint32_t pieces = (flags & 1) ? (count + kFlagPiece - 1) / kFlagPiece : 1u;
    const ull slot = atomicAdd(&w.ctl->fin_count, (ull)pieces);
    for (uint32_t i = 0; i < pieces; i++) {
        if (slot + i >= w.cap_fin) {
            LEY_FAIL(w.err, kErrCapacity);
            return;
        }
        FinTask f;
        f.start = start + (ull)i * kFlagPiece;
        f.count = (flags & 1) ? min(count - i * kFlagPiece, (uint32_t)kFlagPiece) : count;
        f.digit = (uint16_t)digit;
        f.buf = (uint8_t)buf;
        f.flags = (uint8_t)flags;
        w.fin[slot + i] = f;
    }
}

// Appends a bucket to the next level's big list (called by a whole warp with
// the same arguments): its slot and first tile come from one 64-bit atomic,
// so slots and tiles are numbered in the same order; the lanes fill the
// tile-owner table.
__device__ void append_big_warp(const Work& w, int L1, ull start, uint32_t count, int digit,
                                int buf) {
    const int q = L1 & 1, lane = threadIdx.x & 31;
    const uint32_t nt = ceil_div_u64(count, kPassTile);
    ull pk = 0;
    if (lane == 0) pk = atomicAdd(&w.ctl->lvl[L1].big_packed, (1ull << kPackShift) | (ull)nt);
    pk = __shfl_sync(0xffffffffu, pk, 0);
    const ull slot = pk >> kPackShift;
    const ull tb = pk & kPackMask;
    if (slot >= w.cap_seg || tb + nt > w.cap_tiles) {
        if (lane == 0) LEY_FAIL(w.err, kErrCapacity);
        return;
    }
    if (lane == 0) {
        Seg sg;
        sg.start = start;
        sg.count = count;
        sg.digit = (uint16_t)digit;
        sg.buf = (uint8_t)buf;
        sg.pad = 0;
        w.segs[q][slot] = sg;
        w.seg_tile_base[q][slot] = (uint32_t)tb;
        Diff z;
        z.hi = 0;
        z.lo = 0;
        z.pad = 0;
        w.diff[q][slot] = z;
    }
    for (uint32_t i = lane; i < nt; i += 32) w.seg_tile_owner[q][tb + i] = (uint32_t)slot;
}

// One warp per bucket of level L's big list (Algorithm 1's control flow):
//  - a bucket of at most kSmall tuples becomes a finishing task;
//  - a bucket whose current digit is single-valued skips to the first digit
//    where its keys differ, without moving (or finishes if none is left);
//  - otherwise it is scattered this level: its sub-buckets above kSmall
//    recurse on the next digit, runs of smaller ones are packed into
//    finishing tasks of at most kSmall tuples.
__global__ void __launch_bounds__(128)
k_classify(Work w, KeySpec ks, int L) {
    __shared__ uint32_t sh_cnt[4][kRadix];   // per warp: bin counts
    __shared__ uint32_t sh_gs[4][kRadix];    // per warp: task start offsets
    __shared__ uint32_t sh_gc[4][kRadix];    // per warp: count << 1 | single-bucket
    pdl_enter();
    const int p = L & 1, lane = threadIdx.x & 31;
    const ull packed = w.ctl->lvl[L].big_packed;
    const uint32_t nseg = (uint32_t)(packed >> kPackShift);
    if (nseg > w.cap_seg) {
        if (threadIdx.x == 0 && blockIdx.x == 0) LEY_FAIL(w.err, kErrCapacity);
        return;
    }
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < nseg; s += warps) {
        const Seg sg = w.segs[p][s];
        if (lane == 0) w.seg_pass[p][s] = kNoPass;
        if (sg.count <= ks.big) {
            if (lane == 0) emit_fin(w, sg.start, sg.count, sg.digit, sg.buf, 0);
            continue;
        }
        const uint32_t* h = w.hist[p] + (ull)s * kRadix;
        uint32_t c8[8], sum = 0;
        int nz = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            c8[k] = h[lane * 8 + k];
            sum += c8[k];
            nz += c8[k] != 0;
        }
        nz = __reduce_add_sync(0xffffffffu, (uint32_t)nz);
        if (nz <= 1) {
            const Diff df = w.diff[p][s];
            const int d2 = first_varying_digit(df.hi & ks.hi_mask, df.lo & ks.lo_mask,
                                               sg.digit + 1, ks.ndig);
            if (d2 >= ks.ndig) {
                if (lane == 0) emit_fin(w, sg.start, sg.count, ks.ndig, sg.buf, 1);
            } else {
                append_big_warp(w, L + 1, sg.start, sg.count, d2, sg.buf);
            }
            continue;
        }
        ull e = 0;
        if (lane == 0) e = atomicAdd(&w.ctl->lvl[L].pass_count, 1ull);
        e = __shfl_sync(0xffffffffu, e, 0);
        if (e >= w.cap_seg) {
            if (lane == 0) LEY_FAIL(w.err, kErrCapacity);
            continue;
        }
        if (lane == 0) w.seg_pass[p][s] = (uint32_t)e;
        // Exclusive scan over the 256 bins (lane l owns bins 8l..8l+7).
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t off8[8], run = incl - sum;
        uint32_t* bb = w.bucket_base + e * kRadix;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            off8[k] = run;
            bb[lane * 8 + k] = run;
            run += c8[k];
        }
        const int nb = sg.buf ^ 1;
        const int d1 = sg.digit + 1;
        // Big sub-buckets recurse.  The warp reserves list slots and tiles for
        // all of them with one atomic (slot and tile order agree), then each
        // lane writes its own bins' entries and tile owners.
        uint32_t nbig = 0, tbig = 0;
#pragma unroll
        for (int k = 0; k < 8; k++)
            if (c8[k] > ks.big) {
                nbig++;
                tbig += ceil_div_u64(c8[k], kPassTile);
            }
        if (d1 < ks.ndig) {
            uint32_t nb_incl = nbig, tb_incl = tbig;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y1 = __shfl_up_sync(0xffffffffu, nb_incl, o);
                const uint32_t y2 = __shfl_up_sync(0xffffffffu, tb_incl, o);
                if (lane >= o) {
                    nb_incl += y1;
                    tb_incl += y2;
                }
            }
            const uint32_t nb_tot = __shfl_sync(0xffffffffu, nb_incl, 31);
            const uint32_t tb_tot = __shfl_sync(0xffffffffu, tb_incl, 31);
            ull pk0 = 0;
            if (lane == 0 && nb_tot)
                pk0 = atomicAdd(&w.ctl->lvl[L + 1].big_packed,
                                ((ull)nb_tot << kPackShift) | (ull)tb_tot);
            pk0 = __shfl_sync(0xffffffffu, pk0, 0);
            ull slot = (pk0 >> kPackShift) + (nb_incl - nbig);
            ull tile = (pk0 & kPackMask) + (tb_incl - tbig);
            const int q = (L + 1) & 1;
#pragma unroll
            for (int k = 0; k < 8; k++) {
                if (c8[k] <= ks.big) continue;
                const uint32_t nt = ceil_div_u64(c8[k], kPassTile);
                if (slot >= w.cap_seg || tile + nt > w.cap_tiles) {
                    LEY_FAIL(w.err, kErrCapacity);
                    break;
                }
                Seg sgn;
                sgn.start = sg.start + off8[k];
                sgn.count = c8[k];
                sgn.digit = (uint16_t)d1;
                sgn.buf = (uint8_t)nb;
                sgn.pad = 0;
                w.segs[q][slot] = sgn;
                w.seg_tile_base[q][slot] = (uint32_t)tile;
                Diff z;
                z.hi = 0;
                z.lo = 0;
                z.pad = 0;
                w.diff[q][slot] = z;
                for (uint32_t i = 0; i < nt; i++) w.seg_tile_owner[q][tile + i] = (uint32_t)slot;
                slot++;
                tile += nt;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++)
                if (c8[k] > ks.big) emit_fin(w, sg.start + off8[k], c8[k], ks.ndig, nb, 1);
        }
        // Runs of small sub-buckets are packed greedily into finishing tasks
        // (lane 0 walks the bins in shared memory, the warp then reserves all
        // task slots with one atomic and writes them).
        uint32_t* cs = sh_cnt[threadIdx.x >> 5];
#pragma unroll
        for (int k = 0; k < 8; k++) cs[lane * 8 + k] = c8[k];
        __syncwarp();
        uint32_t ng = 0;
        if (lane == 0) {
            uint32_t off = 0, g_start = 0, g_count = 0, g_nb = 0;
            for (int v = 0; v < kRadix; v++) {
                const uint32_t c = cs[v];
                if (c == 0) continue;
                if (c > ks.big || (g_count && g_count + c > ks.big)) {
                    if (g_count) {
                        sh_gs[threadIdx.x >> 5][ng] = g_start;
                        sh_gc[threadIdx.x >> 5][ng] = (g_count << 1) | (g_nb == 1 ? 1u : 0u);
                        ng++;
                    }
                    g_count = 0;
                    g_nb = 0;
                }
                if (c <= ks.big) {
                    if (g_count == 0) g_start = off;
                    g_count += c;
                    g_nb++;
                }
                off += c;
            }
            if (g_count) {
                sh_gs[threadIdx.x >> 5][ng] = g_start;
                sh_gc[threadIdx.x >> 5][ng] = (g_count << 1) | (g_nb == 1 ? 1u : 0u);
                ng++;
            }
        }
        __syncwarp();  // lane 0's task list is visible to the warp
        ng = __shfl_sync(0xffffffffu, ng, 0);
        ull base = 0;
        if (lane == 0 && ng) base = atomicAdd(&w.ctl->fin_count, (ull)ng);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (uint32_t i = lane; i < ng; i += 32) {
            if (base + i >= w.cap_fin) {
                LEY_FAIL(w.err, kErrCapacity);
                break;
            }
            const uint32_t gc = sh_gc[threadIdx.x >> 5][i];
            FinTask f;
            f.start = sg.start + sh_gs[threadIdx.x >> 5][i];
            f.count = gc >> 1;
            f.digit = (uint16_t)((gc & 1u) ? d1 : sg.digit);
            f.buf = (uint8_t)nb;
            f.flags = (gc & 1u) ? 0 : 2;  // 2: sub-buckets of one bucket, in `digit` order
            w.fin[base + i] = f;
        }
        __syncwarp();
    }
}

// Partition mode (one round of Algorithm 1 only): the single top segment is
// scattered on its digit whatever its histogram, and nothing recurses.
__global__ void k_classify_partition(Work w) {
    if (blockIdx.x != 0) return;
    const int d = threadIdx.x;
    if (d == 0) {
        w.ctl->lvl[0].pass_count = 1;
        w.seg_pass[0][0] = 0;
    }
    // exclusive scan of the 256 bucket sizes (one thread: 256 adds)
    if (d == 0) {
        uint32_t off = 0;
        for (int v = 0; v < kRadix; v++) {
            w.bucket_base[v] = off;
            off += w.hist[0][v];
        }
    }
}

// ------------------------------------------------------------------ pass

// One scatter pass of Algorithm 1 over every big bucket scattered at level L
// (ParallelRadixSort): tile t of a bucket writes each of its digit runs to
//   bucket start + bucket_base[digit] + tile offset[digit] (from k_scan),
// after ranking its tuples stably by digit and staging them in shared memory
// so that every run is written contiguously (cache-aware scattering).
// The tuples of tile t of level L's big list (for an L2 prefetch), or none.
__device__ __noinline__ void pass_prefetch_target(const Work& w, int p, uint32_t nseg,
                                                  uint32_t ntiles, uint32_t t,
                                                  const uint4** ptr, uint32_t* bytes) {
    *bytes = 0;
    if (t >= ntiles) return;
    const uint32_t s = w.seg_tile_owner[p][t];
    if (s >= nseg) return;
    const Seg sg = w.segs[p][s];
    const uint32_t tb = w.seg_tile_base[p][s];
    if (t < tb || sg.buf > 1 || sg.start + sg.count > w.n) return;
    const ull off = (ull)(t - tb) * kPassTile;
    if (off >= sg.count) return;
    *ptr = w.tup[sg.buf] + sg.start + off;
    *bytes = (uint32_t)min((ull)kPassTile, sg.count - off) * (uint32_t)sizeof(uint4);
}

__global__ void __launch_bounds__(kPassThreads, 2)
k_pass(Work w, KeySpec ks, int L) {
    extern __shared__ uint4 stage[];                 // kPassTile tuples
    __shared__ uint32_t wcnt[kPassWarps][kRadix];    // per-warp digit counters
    __shared__ uint32_t loc_off[kRadix];
    __shared__ ull gbase[kRadix];
    __shared__ uint32_t scan_tot[kRadix / 32];
    pdl_enter();

    const int p = L & 1;
    const ull packed = w.ctl->lvl[L].big_packed;
    const uint32_t nseg = (uint32_t)(packed >> kPackShift);
    const uint32_t ntiles = (uint32_t)(packed & kPackMask);
    if (ntiles > w.cap_tiles || nseg > w.cap_seg) {
        if (threadIdx.x == 0 && blockIdx.x == 0) LEY_FAIL(w.err, kErrCapacity);
        return;
    }
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt_mask = lanemask_lt();
    // Thread 0 asks the L2 for the CTA's tiles one tile ahead: while tile t
    // is scattered, tile t + grid is being fetched and tile t + 2 grid is
    // looked up in steps (owner, then bucket), so no lookup is waited for.
    const uint4* pf_ptr = nullptr;
    uint32_t pf_bytes = 0;
    if (tid == 0) pass_prefetch_target(w, p, nseg, ntiles, blockIdx.x + gridDim.x, &pf_ptr, &pf_bytes);
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        if (tid == 0 && pf_bytes) l2_prefetch_bulk(pf_ptr, pf_bytes);
        pf_bytes = 0;
        const uint32_t tn = t + 2 * gridDim.x;
        uint32_t sn = kNoPass;
        if (tid == 0 && tn < ntiles) sn = w.seg_tile_owner[p][tn];
        const uint32_t s = w.seg_tile_owner[p][t];
        const uint32_t e = s < nseg ? w.seg_pass[p][s] : kNoPass;
        if (e == kNoPass) continue;  // bucket not scattered at this level
        const Seg sg = w.segs[p][s];
        const uint32_t tile0 = w.seg_tile_base[p][s];
        if (sg.start + sg.count > w.n || t < tile0 || sg.buf > 1 || e >= w.cap_seg) {
            if (tid == 0) LEY_FAIL(w.err, kErrCapacity);  // never for a valid list
            continue;
        }
        __syncthreads();  // previous tile's shared state is no longer read
        for (int i = tid; i < kPassWarps * kRadix; i += kPassThreads) (&wcnt[0][0])[i] = 0;
        const uint32_t lt = t - tile0;
        const ull base = sg.start + (ull)lt * kPassTile;
        const uint32_t m = min((uint32_t)kPassTile, sg.count - lt * (uint32_t)kPassTile);
        const uint4* src = w.tup[sg.buf];
        uint4* dst = w.tup[sg.buf ^ 1];
        const int d = sg.digit;
        ull gb = 0;
        if (tid < kRadix)
            gb = sg.start + w.bucket_base[(ull)e * kRadix + tid] +
                 w.tile_cnt[(ull)t * kRadix + tid];

        // Warp `warp` owns items [warp*256, warp*256+256); item k of a lane
        // is at warp*256 + k*32 + lane, so the k-major order is input order
        // and the ranks below are stable.
        uint4 v[kPassItems];
        uint32_t rd[kPassItems];  // (rank among the warp's items of the digit) << 8 | digit
#pragma unroll
        for (int k = 0; k < kPassItems; k++) {
            uint32_t idx = warp * (kPassItems * 32) + k * 32 + lane;
            v[k] = idx < m ? src[base + idx] : make_uint4(0, 0, 0, 0);
        }
        __syncthreads();  // counters zeroed
#pragma unroll
        for (int k = 0; k < kPassItems; k++) {
            const uint32_t idx = warp * (kPassItems * 32) + k * 32 + lane;
            const bool valid = idx < m;
            const uint32_t dk = valid ? digit_of(v[k], d) : 0u;
            rd[k] = (warp_rank(wcnt[warp], dk, valid, lt_mask, lane) << 8) | dk;
        }
        __syncthreads();
        Seg sgn;
        uint32_t tbn = 0;
        if (tid == 0 && sn < nseg) {
            sgn = w.segs[p][sn];
            tbn = w.seg_tile_base[p][sn];
        }
        uint32_t tile_cnt = 0, incl = 0;
        if (tid < kRadix) {
            // Thread `tid` owns digit tid: exclusive offsets over warps, then
            // the tile-local offset of each digit's run.
            const int dig = tid;
#pragma unroll
            for (int ww = 0; ww < kPassWarps; ww++) {
                const uint32_t c = wcnt[ww][dig];
                wcnt[ww][dig] = tile_cnt;
                tile_cnt += c;
            }
            incl = tile_cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) scan_tot[warp] = incl;
        }
        __syncthreads();
        if (tid < kRadix) {
            uint32_t wp = 0;
#pragma unroll
            for (int ww = 0; ww < kRadix / 32; ww++) wp += ww < warp ? scan_tot[ww] : 0u;
            loc_off[tid] = wp + incl - tile_cnt;
            gbase[tid] = gb;
        }
        __syncthreads();
        // Stage the tile in shared memory in sorted-by-digit order.
#pragma unroll
        for (int k = 0; k < kPassItems; k++) {
            const uint32_t idx = warp * (kPassItems * 32) + k * 32 + lane;
            const uint32_t dk = rd[k] & 0xFFu;
            const uint32_t pos = loc_off[dk] + wcnt[warp][dk] + (rd[k] >> 8);
            if (idx < m) {
                if (pos < (uint32_t)kPassTile) stage[pos] = v[k];
                else LEY_FAIL(w.err, kErrCapacity);  // inconsistent ranks: never
            }
        }
        __syncthreads();
        if (tid == 0 && sn < nseg && tn >= tbn && sgn.buf <= 1 && sgn.start + sgn.count <= w.n) {
            const ull off = (ull)(tn - tbn) * kPassTile;
            if (off < sgn.count) {
                pf_ptr = w.tup[sgn.buf] + sgn.start + off;
                pf_bytes = (uint32_t)min((ull)kPassTile, sgn.count - off) * (uint32_t)sizeof(uint4);
            }
        }
        // Write each digit's run contiguously to its bucket.
        const ull seg_end = sg.start + sg.count;
        for (uint32_t i = tid; i < m; i += kPassThreads) {
            const uint4 tv = stage[i];
            const uint32_t dd = digit_of(tv, d);
            const ull pos = gbase[dd] + (i - loc_off[dd]);
            if (pos >= sg.start && pos < seg_end) dst[pos] = tv;
            else LEY_FAIL(w.err, kErrCapacity);
        }
    }
}

// ---------------------------------------------------------------- finish

template <int MODE>
struct Emitter;

template <>
struct Emitter<0> {  // records: the output permutation
    uint32_t* perm;
    __device__ __forceinline__ void operator()(ull pos, const uint4& t) const { perm[pos] = t.w; }
};
template <>
struct Emitter<1> {  // pairs: sorted keys and their payloads
    uint64_t* keys;
    uint32_t* idx;
    __device__ __forceinline__ void operator()(ull pos, const uint4& t) const {
        keys[pos] = key_hi(t);
        idx[pos] = t.z;
    }
};

template <>
struct Emitter<2> {  // 100-byte records gathered straight into place
    const uint8_t* in;
    uint8_t* out;
    ull n_in;        // records at `in`: every source index is below it
};

// Batched sorts: the task's request is found from its first position
// (tile -> request table), and the task is emitted like a single sort whose
// output arrays are shifted by the request's offset, so that global
// positions index them directly (off is a multiple of kPassTile, so the
// shifted record base keeps the output's 16-byte phase).
template <>
struct Emitter<3> {  // batch of 100-byte records, gathered straight into place
    const BatchReq* reqs;
    const uint32_t* tile_req;
};
template <>
struct Emitter<4> {  // batch of pairs
    const BatchReq* reqs;
    const uint32_t* tile_req;
};

template <int MODE>
struct TaskEmit {
    using type = Emitter<MODE>;
    static constexpr int mode = MODE;
    __device__ static type get(const Emitter<MODE>& e, ull) { return e; }
};
template <>
struct TaskEmit<3> {
    using type = Emitter<2>;
    static constexpr int mode = 2;
    __device__ static type get(const Emitter<3>& e, ull start) {
        const BatchReq q = e.reqs[e.tile_req[start / kPassTile]];
        Emitter<2> t;
        t.in = q.in;
        t.out = q.out - q.off * 100ull;
        t.n_in = q.n;
        return t;
    }
};
template <>
struct TaskEmit<4> {
    using type = Emitter<1>;
    static constexpr int mode = 1;
    __device__ static type get(const Emitter<4>& e, ull start) {
        const BatchReq q = e.reqs[e.tile_req[start / kPassTile]];
        Emitter<1> t;
        t.keys = reinterpret_cast<uint64_t*>(q.out) - q.off;
        t.idx = q.idx_out - q.off;
        return t;
    }
};

// Shared state of one finishing CTA.  B holds the task's tuples; order[j] is
// the position in B of the tuple whose final place in the task is j.
struct FinShared {
    uint32_t cnt[kFinWarps][kRadix];   // per-warp digit counters
    uint16_t off[kFinWarps][kRadix];   // per-warp sub-bucket offsets (warp sorts)
    uint16_t sb_off[kRadix];           // block counting pass: sub-bucket offsets
    uint16_t sb_cnt[kRadix];           //   and sizes
    uint16_t order[kSmall];
    uint32_t q_meta[kFinQueue];        // warp queue: start | count << 16
    uint8_t q_dig[kFinQueue];
    uint8_t q_ready[kFinQueue];
    uint32_t bs_meta[kFinStack];       // block stack (sub-buckets > kWarpMax)
    uint8_t bs_dig[kFinStack];
    int q_head, q_tail, q_pending, bs_n;
    uint32_t warp_tot[kFinWarps];
    uint32_t d3[3];
    uint32_t task;
};

// Rank of tuple tv among the c tuples at B[s..s+c) (strict (key, index) order).
// The order of tup_less, evaluated without branches: every tuple of the
// sub-bucket is compared, so the lanes of a warp stay together.  The whole
// order is one 128-bit unsigned comparison (key bytes 0-7, the key bits of z,
// then the index w, most significant first), taken as the borrow out of a
// four-word subtraction chain.
__device__ __forceinline__ uint32_t cmp_rank(const uint4* B, uint32_t s, uint32_t c,
                                             const uint4& tv, uint32_t lo_mask) {
    const uint32_t vz = tv.z & lo_mask;
    uint32_t r = 0;
#pragma unroll 4
    for (uint32_t j = 0; j < c; j++) {
        const uint4 u = B[s + j];
        uint32_t t, m;
        // borrow out of u - tv over the words (w, z & mask, x, y), least significant first
        asm("sub.cc.u32 %0, %2, %6;\n\t"
            "subc.cc.u32 %0, %3, %7;\n\t"
            "subc.cc.u32 %0, %4, %8;\n\t"
            "subc.cc.u32 %0, %5, %9;\n\t"
            "subc.u32 %1, %10, %10;"
            : "=&r"(t), "=r"(m)
            : "r"(u.w), "r"(u.z & lo_mask), "r"(u.x), "r"(u.y), "r"(tv.w), "r"(vz), "r"(tv.x),
              "r"(tv.y), "r"(0u));
        r -= m;  // m = 0xFFFFFFFF when u < tv
    }
    return r;
}

__device__ __forceinline__ void queue_push(FinShared& S, uint32_t s, uint32_t c, int d,
                                           uint32_t* err) {
    atomicAdd(&S.q_pending, 1);  // counted before it can be claimed
    const int slot = atomicAdd(&S.q_tail, 1);
    if (slot >= kFinQueue) {  // cannot happen (see kFinQueue); report and drop
        LEY_FAIL(err, kErrCapacity);
        atomicSub(&S.q_pending, 1);
        return;
    }
    S.q_meta[slot] = s | (c << 16);
    S.q_dig[slot] = (uint8_t)d;
    __threadfence_block();
    S.q_ready[slot] = 1;
    (void)err;
}

__device__ __forceinline__ void stack_push(FinShared& S, uint32_t s, uint32_t c, int d,
                                           uint32_t* err) {
    const int slot = atomicAdd(&S.bs_n, 1);
    if (slot < kFinStack) {
        S.bs_meta[slot] = s | (c << 16);
        S.bs_dig[slot] = (uint8_t)d;
    } else {
        LEY_FAIL(err, kErrCapacity);
    }
}

// Block-wide stable counting pass on B[r0, r0+c) -- or, with FROM_GLOBAL,
// on the c tuples at gsrc, staged into B[r0, r0+c) -- from digit d0 on
// (SingleThreadRadixSort of Algorithm 1, one CTA instead of one thread).
// Digit d0 is tried first; only when it is the same for every tuple is the
// key-difference mask reduced to find the first digit where keys differ.
// Sub-buckets are finished here by comparison ranking when tiny, else
// queued for a warp (<= kWarpMax) or pushed for the whole CTA.
template <bool FROM_GLOBAL, bool MATCH>
__device__ void fin_block_pass(uint4* B, FinShared& S, const uint4* gsrc, uint32_t r0,
                               uint32_t c, int d0, const KeySpec& ks, uint32_t* err,
                               bool grouped = false) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt_mask = lanemask_lt();
    // Items per thread for this range, so that every warp holds a share:
    // warp w owns items [w * ipt * 32, (w + 1) * ipt * 32) -- contiguous per
    // warp, which keeps the ranks stable.
    const uint32_t ipt = (c + kFinThreads - 1) / kFinThreads;
    const uint32_t wbase = (uint32_t)warp * ipt * 32;
    uint4 v[kFinItems];
    uint32_t rd[kFinItems];
    const uint4 ref = FROM_GLOBAL ? gsrc[0] : B[r0];
#pragma unroll
    for (int k = 0; k < kFinItems; k++) {
        const uint32_t idx = (uint32_t)k < ipt ? wbase + k * 32 + lane : c;
        if (FROM_GLOBAL)
            v[k] = idx < c ? gsrc[idx] : ref;
        else
            v[k] = idx < c ? B[r0 + idx] : ref;
    }
    int ds = d0 < ks.ndig ? d0 : ks.ndig - 1;
    if (FROM_GLOBAL && grouped) {
        // A packed task: whole sub-buckets of one bucket, already in the order
        // of digit ds, so a counting pass would leave every tuple in place.
        // The tuples are staged where they are and each sub-bucket's bounds
        // are found where the digit changes (sb_cnt holds the end until the
        // last step).
        S.sb_cnt[tid] = 0;  // one digit per thread
#pragma unroll
        for (int k = 0; k < kFinItems; k++) {
            const uint32_t idx = (uint32_t)k < ipt ? wbase + k * 32 + lane : c;
            if (idx < c) B[r0 + idx] = v[k];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kFinItems; k++) {
            const uint32_t idx = (uint32_t)k < ipt ? wbase + k * 32 + lane : c;
            if (idx < c) {
                const uint32_t dk = digit_of(v[k], ds);
                if (idx == 0 || digit_of(B[r0 + idx - 1], ds) != dk) S.sb_off[dk] = (uint16_t)idx;
                if (idx + 1 == c || digit_of(B[r0 + idx + 1], ds) != dk)
                    S.sb_cnt[dk] = (uint16_t)(idx + 1);
            }
        }
        __syncthreads();
        if (S.sb_cnt[tid]) S.sb_cnt[tid] = (uint16_t)(S.sb_cnt[tid] - S.sb_off[tid]);
    } else {
    for (;;) {
#pragma unroll
        for (int ww = 0; ww < kFinWarps; ww++) S.cnt[ww][tid] = 0;
        __syncthreads();  // counters zeroed (and, first time, all reads of B done)
#pragma unroll
        for (int k = 0; k < kFinItems; k++) {
            const uint32_t idx = (uint32_t)k < ipt ? wbase + k * 32 + lane : c;
            rd[k] = 0;
            if ((uint32_t)k >= ipt || wbase + k * 32 >= c) continue;  // no item of the warp: skip
            const bool valid = idx < c;
            const uint32_t dk = valid ? digit_of(v[k], ds) : 0u;
            rd[k] = (warp_rank_rw<MATCH>(S.cnt[warp], dk, valid, lt_mask) << 8) | dk;
        }
        __syncthreads();
        {
            const int dig = tid;
            uint32_t run = 0;
#pragma unroll
            for (int ww = 0; ww < kFinWarps; ww++) {
                const uint32_t cc = S.cnt[ww][dig];
                S.cnt[ww][dig] = run;
                run += cc;
            }
            uint32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) S.warp_tot[warp] = incl;
            __syncthreads();
            uint32_t wp = 0;
#pragma unroll
            for (int ww = 0; ww < kFinWarps; ww++) wp += ww < warp ? S.warp_tot[ww] : 0u;
            S.sb_off[dig] = (uint16_t)(wp + incl - run);
            S.sb_cnt[dig] = (uint16_t)run;
        }
        __syncthreads();
        if (S.sb_cnt[digit_of(ref, ds)] != c) break;  // digit ds splits the range
        // Digit ds is the same for every tuple: find where the keys differ.
        if (tid < 3) S.d3[tid] = 0;
        ull dhi = 0;
        uint32_t dlo = 0;
#pragma unroll
        for (int k = 0; k < kFinItems; k++) {
            dhi |= key_hi(v[k]) ^ key_hi(ref);
            dlo |= v[k].z ^ ref.z;
        }
        __syncthreads();
        warp_or_diff(dhi & ks.hi_mask, dlo & ks.lo_mask, S.d3);
        __syncthreads();
        const int d2 = first_varying_digit(((ull)S.d3[0] << 32) | S.d3[1], S.d3[2], ds + 1,
                                           ks.ndig);
        if (d2 >= ks.ndig) {
            // All keys equal: the input order is the answer.
#pragma unroll
            for (int k = 0; k < kFinItems; k++) {
                const uint32_t idx = (uint32_t)k < ipt ? wbase + k * 32 + lane : c;
                if (idx < c) {
                    if (FROM_GLOBAL) B[r0 + idx] = v[k];
                    S.order[r0 + idx] = (uint16_t)(r0 + idx);
                }
            }
            return;
        }
        ds = d2;
        __syncthreads();  // everyone has read sb_cnt and d3 before the next attempt
    }
#pragma unroll
    for (int k = 0; k < kFinItems; k++) {
        const uint32_t idx = (uint32_t)k < ipt ? wbase + k * 32 + lane : c;
        const uint32_t dk = rd[k] & 0xFFu;
        const uint32_t pos = r0 + S.sb_off[dk] + S.cnt[warp][dk] + (rd[k] >> 8);
        if (idx < c) {
            if (pos < r0 + c) B[pos] = v[k];
            else LEY_FAIL(err, kErrCapacity);  // inconsistent ranks: never
        }
    }
    }
    __syncthreads();
    {
        const uint32_t sc = S.sb_cnt[tid];
        const uint32_t s2 = r0 + S.sb_off[tid];
        if (sc > (uint32_t)kWarpMax) stack_push(S, s2, sc, ds + 1, err);
        else if (sc > ks.tiny) queue_push(S, s2, sc, ds + 1, err);
    }
    // Tiny sub-buckets: rank by comparison (ComparisonSort of Algorithm 1).
    for (uint32_t i = tid; i < c; i += kFinThreads) {
        const uint4 tv = B[r0 + i];
        const uint32_t dd = digit_of(tv, ds);
        const uint32_t sc = S.sb_cnt[dd];
        if (sc <= ks.tiny) {
            const uint32_t so = r0 + S.sb_off[dd];
            const uint32_t r = cmp_rank(B, so, sc, tv, ks.lo_mask);
            if (r < sc) S.order[so + r] = (uint16_t)(r0 + i);
            else LEY_FAIL(err, kErrCapacity);  // tv not in its sub-bucket: never
        }
    }
}

// One warp sorts the c <= kWarpMax tuples at B[s, s+c) from digit d0 on:
// a stable counting pass on the first digit where they differ, comparison
// ranking of tiny sub-buckets, and larger ones back onto the queue.
template <bool MATCH>
__device__ void fin_warp_sort(uint4* B, FinShared& S, uint32_t s, uint32_t c, int d0,
                              const KeySpec& ks, uint32_t* err) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt_mask = lanemask_lt();
    uint32_t* cnt = S.cnt[warp];
    uint16_t* off = S.off[warp];
    const uint4 ref = B[s];
    uint4 v[kFinItems];
    uint32_t rd[kFinItems];
    ull dhi = 0;
    uint32_t dlo = 0;
#pragma unroll
    for (int k = 0; k < kFinItems; k++) {
        const uint32_t idx = k * 32 + lane;
        v[k] = idx < c ? B[s + idx] : ref;
        dhi |= key_hi(v[k]) ^ key_hi(ref);
        dlo |= v[k].z ^ ref.z;
    }
    dhi &= ks.hi_mask;
    dlo &= ks.lo_mask;
    const uint32_t a = __reduce_or_sync(0xffffffffu, (uint32_t)(dhi >> 32));
    const uint32_t b = __reduce_or_sync(0xffffffffu, (uint32_t)dhi);
    const uint32_t z = __reduce_or_sync(0xffffffffu, dlo);
    const int ds = first_varying_digit(((ull)a << 32) | b, z, d0, ks.ndig);
    if (ds >= ks.ndig) {
        for (uint32_t i = lane; i < c; i += 32) S.order[s + i] = (uint16_t)(s + i);
        __syncwarp();
        return;
    }
#pragma unroll
    for (int k = 0; k < kRadix / 32; k++) cnt[k * 32 + lane] = 0;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kFinItems; k++) {
        const uint32_t idx = k * 32 + lane;
        rd[k] = 0;
        if (k * 32 >= (int)c) continue;  // no item of the warp: skip
        const bool valid = idx < c;
        const uint32_t dk = valid ? digit_of(v[k], ds) : 0u;
        rd[k] = (warp_rank_rw<MATCH>(cnt, dk, valid, lt_mask) << 8) | dk;
    }
    __syncwarp();
    // Exclusive scan of the 256 counters: lane l owns bins 8l..8l+7.
    uint32_t c8[8], sum = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        c8[k] = cnt[lane * 8 + k];
        sum += c8[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        off[lane * 8 + k] = (uint16_t)run;
        run += c8[k];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kFinItems; k++) {
        const uint32_t idx = k * 32 + lane;
        const uint32_t dk = rd[k] & 0xFFu;
        const uint32_t pos = s + off[dk] + (rd[k] >> 8);
        if (idx < c) {
            if (pos < s + c) B[pos] = v[k];
            else LEY_FAIL(err, kErrCapacity);  // inconsistent ranks: never
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 8; k++)
        if (c8[k] > ks.tiny) queue_push(S, s + off[lane * 8 + k], c8[k], ds + 1, err);
    for (uint32_t i = lane; i < c; i += 32) {
        const uint4 tv = B[s + i];
        const uint32_t dd = digit_of(tv, ds);
        const uint32_t sc = cnt[dd];
        if (sc <= ks.tiny) {
            const uint32_t so = s + off[dd];
            const uint32_t r = cmp_rank(B, so, sc, tv, ks.lo_mask);
            if (r < sc) S.order[so + r] = (uint16_t)(s + i);
            else LEY_FAIL(err, kErrCapacity);  // tv not in its sub-bucket: never
        }
    }
    __syncwarp();
}

// Warps take queued sub-buckets until every queued one is finished
// (the small-bucket queue of Algorithm 1, drained by the CTA's warps).
template <bool MATCH>
__device__ void fin_drain_queue(uint4* B, FinShared& S, const KeySpec& ks, uint32_t* err) {
    const int lane = threadIdx.x & 31;
    uint32_t idle = 0;
    while (true) {
        // Lane 0 claims an entry and reads it; the warp acts on the broadcast.
        int slot = -1, pending = 0;
        uint32_t meta = 0, dg = 0, ok = 1;
        if (lane == 0) {
            const int h = *(volatile int*)&S.q_head;
            const int tl = min(*(volatile int*)&S.q_tail, kFinQueue);
            if (h < tl && atomicCAS(&S.q_head, h, h + 1) == h) {
                slot = h;
                uint32_t spins = 0;
                while (*(volatile uint8_t*)&S.q_ready[slot] == 0) {
                    if (++spins > kSpinLimit) {
                        LEY_FAIL(err, kErrTimeout);
                        ok = 0;
                        break;
                    }
                }
                __threadfence_block();
                meta = *(volatile uint32_t*)&S.q_meta[slot];
                dg = *(volatile uint8_t*)&S.q_dig[slot];
                *(volatile uint8_t*)&S.q_ready[slot] = 0;
            } else {
                pending = *(volatile int*)&S.q_pending;
            }
        }
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (slot >= 0) {
            meta = __shfl_sync(0xffffffffu, meta, 0);
            dg = __shfl_sync(0xffffffffu, dg, 0);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            const uint32_t s0 = meta & 0xFFFFu, c0 = meta >> 16;
            if (ok && s0 + c0 <= (uint32_t)kSmall && c0 <= (uint32_t)kWarpMax)
                fin_warp_sort<MATCH>(B, S, s0, c0, (int)dg, ks, err);
            else if (lane == 0)
                LEY_FAIL(err, kErrCapacity);
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                atomicSub(&S.q_pending, 1);
            }
            idle = 0;
        } else {
            pending = __shfl_sync(0xffffffffu, pending, 0);
            if (pending == 0) break;
            if (++idle > kSpinLimit) {
                if (lane == 0) LEY_FAIL(err, kErrTimeout);
                break;
            }
            __nanosleep(32);
        }
    }
}

// Record gather of one finished task: out[start + j] = in[src index of j]
// for j < count, where the source index is sidx[j] (shared memory), or
// src[j].w when the task's tuples are already in order (flagged).
//
// Each warp owns 32 of B's 112-byte windows and takes rounds of 32 records
// (round r of the task goes to warp r % 8), independently of the other
// warps.  Its lanes copy the records' 16-byte aligned windows as 16-byte
// asynchronous copies (cp.async: many small copies in flight at once), wait
// for their own, shift the 32 records in place into 3200 contiguous output
// bytes, and write them as one bulk store of the 16-byte aligned middle plus
// word stores of the ragged ends.  The output is staged at its own 16-byte
// phase (ph) inside the warp's windows, so the aligned middle is aligned in
// shared memory too.
__device__ void fin_gather_records(uint8_t* Bb, const uint32_t* sidx, const uint4* src,
                                   bool flagged, ull start, uint32_t count, const Emitter<2>& e,
                                   uint32_t* err) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* wreg = Bb + warp * (32 * kWinBytes);  // this warp's 32 windows
    const uint32_t* wsrc = reinterpret_cast<const uint32_t*>(wreg);
    __syncthreads();  // B's previous contents (the task's tuples) are no longer read
    for (uint32_t r0 = (uint32_t)warp * 32; r0 < count; r0 += kFinThreads) {
        const uint32_t nv = min(count - r0, 32u);
        const uint32_t j = r0 + lane;
        uint32_t o = 0;
        ull wsb = 0;  // this lane's record's aligned window (byte offset in the input)
        if (j < count) {
            uint32_t p = flagged ? src[j].w : sidx[j];
            if (p >= e.n_in) {  // never for a valid task list; keeps reads in bounds
                LEY_FAIL(err, kErrCapacity);
                p = 0;
            }
            const ull sb = (ull)p * kRec;
            o = (uint32_t)(sb & 15) >> 2;
            wsb = sb & ~15ull;
        }
        // The 32 windows as 224 16-byte pieces: piece c is part c % 7 of
        // record c / 7; lane l copies pieces l, l + 32, ..., l + 192.
#pragma unroll
        for (int u = 0; u < 7; u++) {
            const uint32_t c = (uint32_t)lane + 32u * u;
            const uint32_t k = c / 7u, part = c - 7u * k;
            const ull kb = __shfl_sync(0xffffffffu, wsb, (int)k);
            if (k < nv)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                             ::"r"(smem_addr(wreg + k * kWinBytes + part * 16)),
                             "l"(e.in + kb + part * 16)
                             : "memory");
        }
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncwarp();  // every lane's pieces have landed
        const uint32_t words = nv * kRecWords;
        const ull g0 = (start + r0) * kRec, g1 = g0 + 4ull * words;
        const uint32_t ph = (uint32_t)(g0 & 15);  // 0, 4, 8 or 12
        uint32_t* wdst = reinterpret_cast<uint32_t*>(wreg + ph);
        // Output word q (record k = q / 25, word i) comes from window word
        // 28k + o_k + i.  Past record 0 the source never lies below the
        // destination by more than the step, and record 0 is copied within
        // the first step, so a forward copy in steps of 128 words (all reads
        // of a step before its writes) is safe in place.
        for (uint32_t q0 = 0; q0 < words; q0 += 128) {
            uint32_t val[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint32_t q = q0 + 32 * u + lane;
                const uint32_t k = q / kRecWords;
                const uint32_t ok = __shfl_sync(0xffffffffu, o, k & 31);
                val[u] = q < words ? wsrc[k * (kWinBytes / 4) + ok + (q - k * kRecWords)] : 0u;
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const uint32_t q = q0 + 32 * u + lane;
                if (q < words) wdst[q] = val[u];
            }
            __syncwarp();
        }
        fence_proxy_async_smem();  // the shifted words are read by the bulk store
        __syncwarp();
        const ull a0 = (g0 + 15) & ~15ull, a1 = g1 & ~15ull;
        uint32_t* outw = reinterpret_cast<uint32_t*>(e.out + g0);
        if (a1 > a0) {
            const uint32_t head = (uint32_t)(a0 - g0) >> 2;
            const uint32_t tail0 = (uint32_t)(a1 - g0) >> 2, tail = words - tail0;
            if ((uint32_t)lane < head) outw[lane] = wdst[lane];
            if (lane >= 8 && (uint32_t)lane - 8 < tail) outw[tail0 + lane - 8] = wdst[tail0 + lane - 8];
            if (lane == 0) {
                tma_store_1d(e.out + a0, reinterpret_cast<uint8_t*>(wdst) + (a0 - g0),
                             (uint32_t)(a1 - a0));
                bulk_commit();
                bulk_wait_read_0();  // the windows are refilled next round
            }
        } else {
            for (uint32_t q = lane; q < words; q += 32) outw[q] = wdst[q];
        }
        __syncwarp();
    }
    __syncthreads();  // B is reused by the next task
}

template <int MODE>
__global__ void __launch_bounds__(kFinThreads, 4)
k_finish(Work w, KeySpec ks, Emitter<MODE> emit) {
    extern __shared__ uint4 B[];  // kSmall tuples
    __shared__ FinShared S;
    pdl_enter();
    const ull nfin = w.ctl->fin_count < w.cap_fin ? w.ctl->fin_count : w.cap_fin;
    const int tid = threadIdx.x;
    constexpr int TM = TaskEmit<MODE>::mode;  // how a task is emitted
    constexpr bool kMatch = TM != 1;          // records: match ranks; pairs: ballots
    for (int i = tid; i < kFinQueue; i += kFinThreads) S.q_ready[i] = 0;
    if (tid == 0) S.task = atomicAdd(&w.ctl->fin_ctr, 1u);
    while (true) {
        __syncthreads();
        const uint32_t ti = S.task;
        if (ti >= nfin) break;
        const FinTask tk = w.fin[ti];
        __syncthreads();  // every thread has read S.task
        // Claim the next task now; its number is needed only at the end.
        uint32_t next = 0;
        if (tid == 0) {
            next = atomicAdd(&w.ctl->fin_ctr, 1u);
            S.q_head = S.q_tail = S.q_pending = S.bs_n = 0;
        }
        bool skip = false;
        if (tk.start + tk.count > w.n || tk.buf > 1 ||
            (!(tk.flags & 1) && tk.count > (uint32_t)kSmall)) {  // never for a valid task list
            if (tid == 0) LEY_FAIL(w.err, kErrCapacity);
            skip = true;
        }
        const uint4* src = w.tup[tk.buf & 1] + tk.start;
        const typename TaskEmit<MODE>::type te = TaskEmit<MODE>::get(emit, tk.start);
        if (!skip && (tk.flags & 1)) {  // all keys equal: input order
            if constexpr (TM == 2) {
                fin_gather_records(reinterpret_cast<uint8_t*>(B), nullptr, src, true, tk.start,
                                   tk.count, te, w.err);
            } else {
                for (uint32_t i = tid; i < tk.count; i += kFinThreads) te(tk.start + i, src[i]);
            }
            skip = true;
        }
        if (!skip) {
            fin_block_pass<true, kMatch>(B, S, src, 0, tk.count, tk.digit, ks, w.err,
                                         (tk.flags & 2) != 0);
            __syncthreads();
            while (S.q_tail != 0 || S.bs_n != 0) {
                fin_drain_queue<kMatch>(B, S, ks, w.err);
                __syncthreads();
                const int ns = S.bs_n;
                if (ns <= 0) break;
                const int top = (ns > kFinStack ? kFinStack : ns) - 1;
                const uint32_t meta = S.bs_meta[top];
                const int dg = S.bs_dig[top];
                __syncthreads();
                if (tid == 0) {
                    S.bs_n = top;
                    S.q_head = S.q_tail = S.q_pending = 0;
                }
                if ((meta & 0xFFFFu) + (meta >> 16) > (uint32_t)kSmall) {
                    if (tid == 0) LEY_FAIL(w.err, kErrCapacity);
                    __syncthreads();
                    continue;
                }
                fin_block_pass<false, kMatch>(B, S, src, meta & 0xFFFFu, meta >> 16, dg, ks, w.err);
                __syncthreads();
            }
            if constexpr (TM == 2) {
                // The task's source indices in final order (count <= kSmall
                // entries over the counters, which are free now), then the
                // records themselves.
                uint32_t* sidx = &S.cnt[0][0];
                for (uint32_t j = tid; j < tk.count; j += kFinThreads) {
                    uint32_t o = S.order[j];
                    if (o >= tk.count) {  // a position left unset: report, stay in bounds
                        LEY_FAIL(w.err, kErrCapacity);
                        o = 0;
                    }
                    sidx[j] = B[o].w;
                }
                fin_gather_records(reinterpret_cast<uint8_t*>(B), sidx, src, false, tk.start,
                                   tk.count, te, w.err);
            } else {
                // Coalesced write of the task's final order.
                for (uint32_t j = tid; j < tk.count; j += kFinThreads) {
                    uint32_t o = S.order[j];
                    if (o >= tk.count) {  // a position left unset: report, stay in bounds
                        LEY_FAIL(w.err, kErrCapacity);
                        o = 0;
                    }
                    te(tk.start + j, B[o]);
                }
            }
        }
        __syncthreads();
        if (tid == 0) S.task = next;
    }
}

// --------------------------------------------------------- partition out

__global__ void k_partition_out(Work w, ull n, uint32_t* order_out, ull* hist_out) {
    const uint4* t = w.tup[1];
    for (ull i = (ull)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (ull)gridDim.x * blockDim.x)
        order_out[i] = t[i].w;
    if (blockIdx.x == 0) hist_out[threadIdx.x] = w.hist[0][threadIdx.x];
}

// -------------------------------------------------------------- launchers
cudaError_t launch_extract_window(const LaunchCfg& c, const uint8_t* in, const uint32_t* order,
                                  ull n, uint32_t rec, uint32_t koff, KeySpec ks, const Work& w) {
    const int grid = (int)min((uint32_t)c.grid, ceil_div_u64(n, kPassTile));
    k_extract_window<<<grid, 256, 0, c.stream>>>(in, order, n, rec, koff, ks, w, w.err);
    return cudaGetLastError();
}

cudaError_t launch_compose_order(cudaStream_t s, int grid, const uint32_t* order,
                                 const uint32_t* pass, uint32_t* next, ull n, uint32_t* err) {
    k_compose_order<<<grid, 256, 0, s>>>(order, pass, next, n, err);
    return cudaGetLastError();
}

cudaError_t launch_batch_setup(cudaStream_t s, const BatchReq* reqs, uint32_t R, const Work& w,
                               uint32_t* tile_req, uint32_t ntiles, int digit0) {
    k_batch_setup<<<(R + 255) / 256, 256, 0, s>>>(reqs, R, w, ntiles, digit0);
    if (cudaGetLastError() != cudaSuccess) return cudaErrorLaunchFailure;
    k_batch_tiles<<<(ntiles + 255) / 256, 256, 0, s>>>(reqs, R, w, tile_req, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_batch_extract_records(const LaunchCfg& c, const BatchReq* reqs,
                                         const uint32_t* tile_req, uint32_t ntiles, uint32_t rec,
                                         KeySpec ks, const Work& w) {
    const int grid = (int)min((uint32_t)c.grid, ntiles);
    if (rec == 100)
        k_batch_extract_records<100><<<grid, 256, 0, c.stream>>>(reqs, tile_req, ntiles, rec, ks, w, 0);
    else
        k_batch_extract_records<0><<<grid, 256, 0, c.stream>>>(reqs, tile_req, ntiles, rec, ks, w, 0);
    return cudaGetLastError();
}

cudaError_t launch_batch_extract_pairs(const LaunchCfg& c, const BatchReq* reqs,
                                       const uint32_t* tile_req, uint32_t ntiles, const Work& w) {
    const int grid = (int)min((uint32_t)c.grid, ntiles);
    k_batch_extract_pairs<<<grid, 256, 0, c.stream>>>(reqs, tile_req, ntiles, w);
    return cudaGetLastError();
}

cudaError_t launch_batch_finish(const LaunchCfg& c, const Work& w, KeySpec ks,
                                const BatchReq* reqs, const uint32_t* tile_req, bool pairs) {
    if (pairs) {
        Emitter<4> e;
        e.reqs = reqs;
        e.tile_req = tile_req;
        return launch_pdl(k_finish<4>, c.grid, kFinThreads, c.smem, c.stream, w, ks, e);
    }
    Emitter<3> e;
    e.reqs = reqs;
    e.tile_req = tile_req;
    return launch_pdl(k_finish<3>, c.grid, kFinThreads, c.smem, c.stream, w, ks, e);
}

cudaError_t launch_batch_gather_generic(cudaStream_t s, int grid, const BatchReq* reqs,
                                        const uint32_t* tile_req, const uint32_t* perm, ull npos,
                                        uint32_t rec, uint32_t* err) {
    k_batch_gather_generic<<<grid, 256, 0, s>>>(reqs, tile_req, perm, npos, rec, err);
    return cudaGetLastError();
}

cudaError_t launch_extract_records(const LaunchCfg& c, const uint8_t* in, ull n, uint32_t rec,
                                   KeySpec ks, const Work& w, int hist_digit) {
    return launch_extract_records_tiles(c, in, n, rec, ks, w, hist_digit, 0,
                                        ceil_div_u64(n, kPassTile));
}

cudaError_t launch_extract_records_tiles(const LaunchCfg& c, const uint8_t* in, ull n,
                                         uint32_t rec, KeySpec ks, const Work& w, int hist_digit,
                                         uint32_t t_begin, uint32_t t_end, const uint8_t* ref_in) {
    if (t_end <= t_begin) return cudaSuccess;
    if (!ref_in) ref_in = in;
    const int grid = (int)min((uint32_t)c.grid, t_end - t_begin);
    if (rec == 100)
        k_extract_records<100><<<grid, 256, 0, c.stream>>>(in, n, rec, ks, w, hist_digit, t_begin,
                                                           t_end, ref_in);
    else
        k_extract_records<0><<<grid, 256, 0, c.stream>>>(in, n, rec, ks, w, hist_digit, t_begin,
                                                         t_end, ref_in);
    return cudaGetLastError();
}

cudaError_t launch_extract_pairs(const LaunchCfg& c, const uint64_t* keys, const uint32_t* idx,
                                 ull n, KeySpec, const Work& w) {
    k_extract_pairs<<<c.grid, 256, 0, c.stream>>>(keys, idx, n, w);
    return cudaGetLastError();
}

cudaError_t launch_init(cudaStream_t s, const Work& w, ull n, int digit0) {
    k_init<<<1, 32, 0, s>>>(w, n, digit0);
    return cudaGetLastError();
}

cudaError_t launch_hist(const LaunchCfg& c, const Work& w, KeySpec ks, int level) {
    return launch_pdl(k_hist, c.grid, kHistThreads, 0, c.stream, w, ks, level);
}

cudaError_t launch_scan(const LaunchCfg& c, const Work& w, int level) {
    return launch_pdl(k_scan, c.grid, kRadix, 0, c.stream, w, level);
}

cudaError_t launch_classify(const LaunchCfg& c, const Work& w, KeySpec ks, int level) {
    return launch_pdl(k_classify, c.grid, 128, 0, c.stream, w, ks, level);
}

cudaError_t launch_classify_partition(cudaStream_t s, const Work& w) {
    k_classify_partition<<<1, 32, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_pass(const LaunchCfg& c, const Work& w, KeySpec ks, int level) {
    return launch_pdl(k_pass, c.grid, kPassThreads, c.smem, c.stream, w, ks, level);
}

cudaError_t launch_finish_records(const LaunchCfg& c, const Work& w, KeySpec ks) {
    Emitter<0> e;
    e.perm = w.perm;
    return launch_pdl(k_finish<0>, c.grid, kFinThreads, c.smem, c.stream, w, ks, e);
}

cudaError_t launch_finish_gather(const LaunchCfg& c, const Work& w, KeySpec ks, const uint8_t* in,
                                 uint8_t* out, ull n_in) {
    Emitter<2> e;
    e.in = in;
    e.out = out;
    e.n_in = n_in;
    return launch_pdl(k_finish<2>, c.grid, kFinThreads, c.smem, c.stream, w, ks, e);
}

cudaError_t launch_finish_pairs(const LaunchCfg& c, const Work& w, KeySpec ks, uint64_t* keys_out,
                                uint32_t* idx_out) {
    Emitter<1> e;
    e.keys = keys_out;
    e.idx = idx_out;
    return launch_pdl(k_finish<1>, c.grid, kFinThreads, c.smem, c.stream, w, ks, e);
}

cudaError_t launch_partition_out(cudaStream_t s, int grid, const Work& w, ull n,
                                 uint32_t* order_out, ull* hist_out) {
    k_partition_out<<<grid, 256, 0, s>>>(w, n, order_out, hist_out);
    return cudaGetLastError();
}

// Shared-memory needs and occupancy of the persistent kernels.
static int g_bps[KK_COUNT];
static bool g_bps_init = false;

size_t kernel_smem(KernelKind k) {
    switch (k) {
        case KK_PASS: return (size_t)kPassTile * sizeof(uint4);
        case KK_FINISH_REC:
        case KK_FINISH_PAIRS:
        case KK_FINISH_GATHER: return (size_t)kSmall * sizeof(uint4);
        default: return 0;
    }
}

int kernel_threads(KernelKind k) {
    switch (k) {
        case KK_PASS: return kPassThreads;
        case KK_HIST: return kHistThreads;
        case KK_FINISH_REC:
        case KK_FINISH_PAIRS:
        case KK_FINISH_GATHER: return kFinThreads;
        default: return 256;
    }
}

int gather_blocks_per_sm(KernelKind k);  // ley_gather.cu

int blocks_per_sm(KernelKind k) {
    if (!g_bps_init) {
        int v = 0;
        cudaFuncSetAttribute(k_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kernel_smem(KK_PASS));
        cudaFuncSetAttribute(k_finish<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kernel_smem(KK_FINISH_REC));
        cudaFuncSetAttribute(k_finish<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kernel_smem(KK_FINISH_PAIRS));
        cudaFuncSetAttribute(k_finish<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kernel_smem(KK_FINISH_GATHER));
        cudaFuncSetAttribute(k_finish<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kernel_smem(KK_FINISH_GATHER));
        cudaFuncSetAttribute(k_finish<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kernel_smem(KK_FINISH_PAIRS));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_extract_records<100>, 256, 0);
        g_bps[KK_EXTRACT_REC] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_extract_pairs, 256, 0);
        g_bps[KK_EXTRACT_PAIRS] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_hist, kHistThreads, 0);
        g_bps[KK_HIST] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_scan, kRadix, 0);
        g_bps[KK_SCAN] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_pass, kPassThreads,
                                                      kernel_smem(KK_PASS));
        g_bps[KK_PASS] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_finish<0>, kFinThreads,
                                                      kernel_smem(KK_FINISH_REC));
        g_bps[KK_FINISH_REC] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_finish<1>, kFinThreads,
                                                      kernel_smem(KK_FINISH_PAIRS));
        g_bps[KK_FINISH_PAIRS] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_finish<2>, kFinThreads,
                                                      kernel_smem(KK_FINISH_GATHER));
        g_bps[KK_FINISH_GATHER] = v > 0 ? v : 1;
        g_bps[KK_GATHER100] = gather_blocks_per_sm(KK_GATHER100);
        g_bps[KK_GATHER100_TMA] = gather_blocks_per_sm(KK_GATHER100_TMA);
        g_bps[KK_GATHER_GENERIC] = gather_blocks_per_sm(KK_GATHER_GENERIC);
        g_bps_init = true;
    }
    return g_bps[k];
}

}  // namespace ley
