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
//                 Algorithm 1), and emits the final permutation.
#include "ley_kernels.h"

namespace ley {

using ull = unsigned long long;

// ------------------------------------------------------------- helpers

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

// Largest i in [0, cnt) with base[i] <= t (base is non-decreasing, base[0] = 0).
__device__ __forceinline__ uint32_t find_owner(const uint32_t* base, uint32_t cnt, uint32_t t) {
    uint32_t lo = 0, hi = cnt;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (base[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
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
                                                 uint32_t rec_rt, uint32_t kb, const KeySpec& ks) {
    const uint32_t rec = REC ? (uint32_t)REC : rec_rt;
    ull s = i * rec;
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

// Histogram update with warp-level aggregation: lanes holding the same digit
// elect one leader that adds the group's size (digit 256 = no item).
__device__ __forceinline__ void hist_add_warp(uint32_t* sh_hist, uint32_t dg) {
    uint32_t peers = __match_any_sync(0xffffffffu, dg);
    if (dg < 256u && (threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1))
        atomicAdd(&sh_hist[dg], (uint32_t)__popc(peers));
}

// ------------------------------------------------------------- extract

template <int REC>
__global__ void __launch_bounds__(256)
k_extract_records(const uint8_t* __restrict__ in, ull n, uint32_t rec_rt, KeySpec ks,
                  uint4* __restrict__ tup, uint32_t* __restrict__ hist0, Diff* __restrict__ diff0,
                  int hist_digit) {
    __shared__ uint32_t sh_hist[kRadix];
    __shared__ uint32_t sh_d[3];
    sh_hist[threadIdx.x] = 0;
    if (threadIdx.x < 3) sh_d[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t kb = (uint32_t)ks.ndig;
    const uint4 ref = load_record_key<REC>(in, 0, rec_rt, kb, ks);
    ull dhi = 0;
    uint32_t dlo = 0;
    constexpr int U = 4;
    const ull stride = (ull)gridDim.x * blockDim.x;
    for (ull base = (ull)blockIdx.x * blockDim.x; base < n; base += stride * U) {
        uint4 t[U];
        bool valid[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            ull i = base + u * stride + threadIdx.x;
            valid[u] = i < n;
            t[u] = valid[u] ? load_record_key<REC>(in, i, rec_rt, kb, ks) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            ull i = base + u * stride + threadIdx.x;
            uint32_t dg = 256u;
            if (valid[u]) {
                t[u].w = (uint32_t)i;
                tup[i] = t[u];
                dg = digit_of(t[u], hist_digit);
                dhi |= key_hi(t[u]) ^ key_hi(ref);
                dlo |= t[u].z ^ ref.z;
            }
            hist_add_warp(sh_hist, dg);
        }
    }
    warp_or_diff(dhi, dlo, sh_d);
    __syncthreads();
    if (sh_hist[threadIdx.x]) atomicAdd(&hist0[threadIdx.x], sh_hist[threadIdx.x]);
    if (threadIdx.x == 0) flush_diff(sh_d, diff0);
}

__global__ void __launch_bounds__(256)
k_extract_pairs(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ idx, ull n,
                uint4* __restrict__ tup, uint32_t* __restrict__ hist0, Diff* __restrict__ diff0) {
    __shared__ uint32_t sh_hist[kRadix];
    __shared__ uint32_t sh_d[3];
    sh_hist[threadIdx.x] = 0;
    if (threadIdx.x < 3) sh_d[threadIdx.x] = 0;
    __syncthreads();
    const ull ref = __ldg(keys);
    ull dhi = 0;
    constexpr int U = 4;
    const ull stride = (ull)gridDim.x * blockDim.x;
    for (ull base = (ull)blockIdx.x * blockDim.x; base < n; base += stride * U) {
        ull k[U];
        uint32_t v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            ull i = base + u * stride + threadIdx.x;
            k[u] = i < n ? __ldg(keys + i) : 0ull;
            v[u] = i < n ? __ldg(idx + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            ull i = base + u * stride + threadIdx.x;
            uint32_t dg = 256u;
            if (i < n) {
                tup[i] = make_uint4((uint32_t)k[u], (uint32_t)(k[u] >> 32), v[u], (uint32_t)i);
                dg = (uint32_t)(k[u] >> 56);
                dhi |= k[u] ^ ref;
            }
            hist_add_warp(sh_hist, dg);
        }
    }
    warp_or_diff(dhi, 0u, sh_d);
    __syncthreads();
    if (sh_hist[threadIdx.x]) atomicAdd(&hist0[threadIdx.x], sh_hist[threadIdx.x]);
    if (threadIdx.x == 0) flush_diff(sh_d, diff0);
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

__global__ void __launch_bounds__(kPassThreads)
k_hist(Work w, KeySpec ks, int L) {
    __shared__ uint32_t sh_hist[kRadix];
    __shared__ uint32_t sh_d[3];
    __shared__ uint32_t sh_tile;
    const int p = L & 1;
    const ull packed = w.ctl->lvl[L].big_packed;
    const uint32_t nseg = (uint32_t)(packed >> kPackShift);
    const uint32_t ntiles = (uint32_t)(packed & kPackMask);
    const int tid = threadIdx.x;
    if (nseg > w.cap_seg) {  // an append overflowed: the list is not usable
        if (tid == 0 && blockIdx.x == 0) atomicOr(w.err, kErrCapacity);
        return;
    }
    while (true) {
        __syncthreads();
        if (tid == 0) sh_tile = atomicAdd(&w.ctl->lvl[L].hist_tile_ctr, 1u);
        sh_hist[tid] = 0;
        if (tid < 3) sh_d[tid] = 0;
        __syncthreads();
        const uint32_t t = sh_tile;
        if (t >= ntiles) break;
        const uint32_t s = find_owner(w.seg_tile_base[p], nseg, t);
        const Seg sg = w.segs[p][s];
        const uint32_t lt = t - w.seg_tile_base[p][s];
        const ull base = sg.start + (ull)lt * kPassTile;
        const uint32_t m = min((uint32_t)kPassTile, sg.count - lt * (uint32_t)kPassTile);
        const uint4* src = w.tup[sg.buf];
        const uint4 ref = src[sg.start];
        uint4 v[kPassItems];
#pragma unroll
        for (int k = 0; k < kPassItems; k++) {
            uint32_t idx = k * kPassThreads + tid;
            v[k] = idx < m ? src[base + idx] : make_uint4(0, 0, 0, 0);
        }
        ull dhi = 0;
        uint32_t dlo = 0;
#pragma unroll
        for (int k = 0; k < kPassItems; k++) {
            uint32_t idx = k * kPassThreads + tid;
            uint32_t dg = 256u;
            if (idx < m) {
                dg = digit_of(v[k], sg.digit);
                dhi |= key_hi(v[k]) ^ key_hi(ref);
                dlo |= (v[k].z ^ ref.z) & ks.lo_mask;
            }
            hist_add_warp(sh_hist, dg);
        }
        warp_or_diff(dhi & ks.hi_mask, dlo, sh_d);
        __syncthreads();
        if (sh_hist[tid]) atomicAdd(&w.hist[p][(ull)s * kRadix + tid], sh_hist[tid]);
        if (tid == 0) flush_diff(sh_d, &w.diff[p][s]);
    }
}

// ------------------------------------------------------------- classify

__device__ void emit_fin(const Work& w, ull start, uint32_t count, int digit, int buf, int flags) {
    ull slot = atomicAdd(&w.ctl->fin_count, 1ull);
    if (slot >= w.cap_fin) {
        atomicOr(w.err, kErrCapacity);
        return;
    }
    FinTask f;
    f.start = start;
    f.count = count;
    f.digit = (uint16_t)digit;
    f.buf = (uint8_t)buf;
    f.flags = (uint8_t)flags;
    w.fin[slot] = f;
}

__device__ void append_big(const Work& w, int L1, ull start, uint32_t count, int digit, int buf) {
    const int q = L1 & 1;
    ull pk = atomicAdd(&w.ctl->lvl[L1].big_packed,
                       (1ull << kPackShift) | (ull)ceil_div_u64(count, kPassTile));
    ull slot = pk >> kPackShift;
    if (slot >= w.cap_seg) {
        atomicOr(w.err, kErrCapacity);
        return;
    }
    Seg s;
    s.start = start;
    s.count = count;
    s.digit = (uint16_t)digit;
    s.buf = (uint8_t)buf;
    s.pad = 0;
    w.segs[q][slot] = s;
    w.seg_tile_base[q][slot] = (uint32_t)(pk & kPackMask);
    uint4* h = reinterpret_cast<uint4*>(w.hist[q] + slot * kRadix);
    for (int i = 0; i < kRadix / 4; i++) h[i] = make_uint4(0, 0, 0, 0);
    Diff z;
    z.hi = 0;
    z.lo = 0;
    z.pad = 0;
    w.diff[q][slot] = z;
}

__global__ void __launch_bounds__(128)
k_classify(Work w, KeySpec ks, int L) {
    const int p = L & 1;
    const ull packed = w.ctl->lvl[L].big_packed;
    const uint32_t nseg = (uint32_t)(packed >> kPackShift);
    if (nseg > w.cap_seg) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(w.err, kErrCapacity);
        return;
    }
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        const Seg sg = w.segs[p][s];
        if (sg.count <= (uint32_t)kSmall) {
            emit_fin(w, sg.start, sg.count, sg.digit, sg.buf, 0);
            continue;
        }
        const uint4* h4 = reinterpret_cast<const uint4*>(w.hist[p] + (ull)s * kRadix);
        int nz = 0;
        for (int i = 0; i < kRadix / 4; i++) {
            uint4 c = h4[i];
            nz += (c.x != 0) + (c.y != 0) + (c.z != 0) + (c.w != 0);
        }
        if (nz <= 1) {
            // The digit is the same across the bucket: skip it without moving
            // anything, straight to the first digit where keys differ.
            const Diff df = w.diff[p][s];
            int d2 = first_varying_digit(df.hi & ks.hi_mask, df.lo & ks.lo_mask, sg.digit + 1,
                                         ks.ndig);
            if (d2 >= ks.ndig)
                emit_fin(w, sg.start, sg.count, ks.ndig, sg.buf, 1);
            else
                append_big(w, L + 1, sg.start, sg.count, d2, sg.buf);
            continue;
        }
        ull pk = atomicAdd(&w.ctl->lvl[L].pass_packed,
                           (1ull << kPackShift) | (ull)ceil_div_u64(sg.count, kPassTile));
        const uint32_t e = (uint32_t)(pk >> kPackShift);
        if (e >= w.cap_seg) {
            atomicOr(w.err, kErrCapacity);
            continue;
        }
        w.pass_slot[e] = s;
        w.pass_tile_base[e] = (uint32_t)(pk & kPackMask);
        uint32_t* bb = w.bucket_base + (ull)e * kRadix;
        const uint32_t* h = w.hist[p] + (ull)s * kRadix;
        const int nb = sg.buf ^ 1;
        const int d1 = sg.digit + 1;
        uint32_t off = 0, g_start = 0, g_count = 0, g_nb = 0;
        for (int v = 0; v < kRadix; v++) {
            const uint32_t c = h[v];
            bb[v] = off;
            if (c == 0) continue;
            if (c > (uint32_t)kSmall) {
                if (g_count) {
                    emit_fin(w, sg.start + g_start, g_count, g_nb == 1 ? d1 : sg.digit, nb, 0);
                    g_count = 0;
                    g_nb = 0;
                }
                if (d1 < ks.ndig)
                    append_big(w, L + 1, sg.start + off, c, d1, nb);
                else
                    emit_fin(w, sg.start + off, c, ks.ndig, nb, 1);
            } else {
                if (g_count && g_count + c > (uint32_t)kSmall) {
                    emit_fin(w, sg.start + g_start, g_count, g_nb == 1 ? d1 : sg.digit, nb, 0);
                    g_count = 0;
                    g_nb = 0;
                }
                if (g_count == 0) g_start = off;
                g_count += c;
                g_nb++;
            }
            off += c;
        }
        if (g_count) emit_fin(w, sg.start + g_start, g_count, g_nb == 1 ? d1 : sg.digit, nb, 0);
    }
}

// Partition mode (one round of Algorithm 1 only): the single top segment is
// scattered on its digit whatever its histogram, and nothing recurses.
__global__ void k_classify_partition(Work w) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const Seg sg = w.segs[0][0];
    w.ctl->lvl[0].pass_packed = (1ull << kPackShift) | ceil_div_u64(sg.count, kPassTile);
    w.pass_slot[0] = 0;
    w.pass_tile_base[0] = 0;
    uint32_t off = 0;
    for (int v = 0; v < kRadix; v++) {
        w.bucket_base[v] = off;
        off += w.hist[0][v];
    }
}

// ------------------------------------------------------------------ pass

constexpr ull kFlagAgg = 1ull << 62;
constexpr ull kFlagInc = 2ull << 62;
constexpr ull kValMask = (1ull << 56) - 1;

__device__ __forceinline__ ull pack_status(ull flag, int epoch, ull val) {
    return flag | ((ull)epoch << 56) | (val & kValMask);
}

__global__ void __launch_bounds__(kPassThreads, 2)
k_pass(Work w, KeySpec ks, int L) {
    extern __shared__ uint4 stage[];                 // kPassTile tuples
    __shared__ uint16_t wcnt[kPassThreads / 32][kRadix];
    __shared__ uint32_t loc_off[kRadix];
    __shared__ ull gbase[kRadix];
    __shared__ uint32_t warp_tot[kPassThreads / 32];
    __shared__ uint32_t sh_tile;
    __shared__ int sh_bad;

    const int p = L & 1;
    const ull pk = w.ctl->lvl[L].pass_packed;
    const uint32_t npass = (uint32_t)(pk >> kPackShift);
    const uint32_t ntiles = (uint32_t)(pk & kPackMask);
    if (ntiles > w.cap_tiles || npass > w.cap_seg) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicOr(w.err, kErrCapacity);
        return;
    }
    const int epoch = L + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt_mask = lanemask_lt();

    while (true) {
        __syncthreads();
        if (tid == 0) {
            sh_tile = atomicAdd(&w.ctl->lvl[L].pass_tile_ctr, 1u);
            sh_bad = 0;
        }
#pragma unroll
        for (int ww = 0; ww < kPassThreads / 32; ww++) wcnt[ww][tid] = 0;
        __syncthreads();
        const uint32_t t = sh_tile;
        if (t >= ntiles) break;
        const uint32_t e = find_owner(w.pass_tile_base, npass, t);
        const uint32_t tile0 = w.pass_tile_base[e];
        const Seg sg = w.segs[p][w.pass_slot[e]];
        const uint32_t lt = t - tile0;
        const ull base = sg.start + (ull)lt * kPassTile;
        const uint32_t m = min((uint32_t)kPassTile, sg.count - lt * (uint32_t)kPassTile);
        const uint4* src = w.tup[sg.buf];
        uint4* dst = w.tup[sg.buf ^ 1];
        const int d = sg.digit;

        // Load: warp `warp` owns items [warp*512, warp*512+512), item k of a
        // lane at warp*512 + k*32 + lane (coalesced, and k-major order is the
        // input order, which keeps the ranks stable).
        // rd[k] = (rank of item k among the warp's items of its digit) << 16
        //        | digit (256 = no item).
        uint4 v[kPassItems];
        uint32_t rd[kPassItems];
#pragma unroll
        for (int k = 0; k < kPassItems; k++) {
            uint32_t idx = warp * (kPassItems * 32) + k * 32 + lane;
            v[k] = idx < m ? src[base + idx] : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int k = 0; k < kPassItems; k++) {
            uint32_t idx = warp * (kPassItems * 32) + k * 32 + lane;
            const uint32_t dk = idx < m ? digit_of(v[k], d) : 256u;
            uint32_t peers = __match_any_sync(0xffffffffu, dk);
            uint32_t cnt = dk < 256u ? wcnt[warp][dk] : 0u;
            rd[k] = ((cnt + __popc(peers & lt_mask)) << 16) | dk;
            __syncwarp();
            if (dk < 256u && lane == __ffs(peers) - 1)
                wcnt[warp][dk] = (uint16_t)(cnt + __popc(peers));
            __syncwarp();
        }
        __syncthreads();

        // Thread `tid` owns digit tid: exclusive offsets over warps, then the
        // tile's count is published for the look-back of later tiles.
        const int dig = tid;
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kPassThreads / 32; ww++) {
            uint32_t c = wcnt[ww][dig];
            wcnt[ww][dig] = (uint16_t)run;
            run += c;
        }
        const uint32_t tile_cnt = run;
        ull* my = w.status + (ull)t * kRadix + dig;
        ull excl = 0;
        if (lt == 0) {
            st_relaxed(my, pack_status(kFlagInc, epoch, tile_cnt));
        } else {
            st_relaxed(my, pack_status(kFlagAgg, epoch, tile_cnt));
            // Decoupled look-back (Merrill & Garland): walk predecessors of
            // this bucket, summing aggregates until an inclusive prefix.
            uint32_t j = t - 1;
            uint32_t spins = 0;
            while (true) {
                ull s = ld_relaxed(w.status + (ull)j * kRadix + dig);
                int ep = (int)((s >> 56) & 0x3F);
                ull flag = s & (3ull << 62);
                if (ep != epoch || flag == 0) {
                    if (++spins > kSpinLimit) {
                        atomicOr(w.err, kErrTimeout);
                        sh_bad = 1;
                        break;
                    }
                    if (spins > 32) __nanosleep(64);
                    continue;
                }
                excl += s & kValMask;
                if (flag == kFlagInc || j == tile0) break;
                j--;
            }
            st_relaxed(my, pack_status(kFlagInc, epoch, excl + tile_cnt));
        }
        // Block exclusive scan of the tile's digit counts: local offsets.
        uint32_t incl = tile_cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        uint32_t wp = 0;
#pragma unroll
        for (int ww = 0; ww < kPassThreads / 32; ww++) wp += ww < warp ? warp_tot[ww] : 0u;
        loc_off[dig] = wp + incl - tile_cnt;
        gbase[dig] = sg.start + w.bucket_base[(ull)e * kRadix + dig] + excl;
        __syncthreads();

        // Stage the tile in shared memory in sorted-by-digit order.
#pragma unroll
        for (int k = 0; k < kPassItems; k++) {
            const uint32_t dk = rd[k] & 0xFFFFu;
            if (dk < 256u) stage[loc_off[dk] + wcnt[warp][dk] + (rd[k] >> 16)] = v[k];
        }
        __syncthreads();
        if (sh_bad) continue;
        // Write each digit's run contiguously to its bucket.
        const ull seg_end = sg.start + sg.count;
        for (uint32_t i = tid; i < m; i += kPassThreads) {
            uint4 tv = stage[i];
            uint32_t dd = digit_of(tv, d);
            ull pos = gbase[dd] + (i - loc_off[dd]);
            if (pos >= sg.start && pos < seg_end) dst[pos] = tv;
            else atomicOr(w.err, kErrCapacity);
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

struct FinShared {
    uint16_t wcnt[kFinThreads / 32][kRadix];
    uint16_t sb_off[kRadix];
    uint16_t sb_cnt[kRadix];
    uint32_t stk_s[kFinStack];
    uint32_t stk_c[kFinStack];
    uint32_t warp_tot[kFinThreads / 32];
    uint32_t d3[3];
    int stk_n;
    uint32_t task;
};

// Sorts B[r0, r0+c) (or, when gsrc != nullptr, the c tuples at gsrc, staged
// into B[0, c)) by key from digit d0 on.  Sub-buckets of at most kTiny tuples
// are finished by comparison ranking; larger ones are pushed on the CTA's
// stack.  Every finished tuple is emitted at out_base + its final position.
template <int MODE>
__device__ void fin_range(uint4* B, FinShared& S, const uint4* gsrc, uint32_t r0, uint32_t c,
                          int d0, const KeySpec& ks, const Emitter<MODE>& emit, ull out_base,
                          uint32_t* err) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt_mask = lanemask_lt();
    uint4 v[kFinItems];
    uint32_t dg[kFinItems], rk[kFinItems];
    if (tid < 3) S.d3[tid] = 0;
#pragma unroll
    for (int ww = 0; ww < kFinThreads / 32; ww++) S.wcnt[ww][tid] = 0;
    const uint4 ref = gsrc ? gsrc[0] : B[r0];
#pragma unroll
    for (int k = 0; k < kFinItems; k++) {
        uint32_t idx = warp * (kFinItems * 32) + k * 32 + lane;
        v[k] = idx < c ? (gsrc ? gsrc[idx] : B[r0 + idx]) : ref;
    }
    ull dhi = 0;
    uint32_t dlo = 0;
#pragma unroll
    for (int k = 0; k < kFinItems; k++) {
        dhi |= key_hi(v[k]) ^ key_hi(ref);
        dlo |= v[k].z ^ ref.z;
    }
    __syncthreads();  // S.d3 / wcnt zeroed, all reads of B done
    warp_or_diff(dhi & ks.hi_mask, dlo & ks.lo_mask, S.d3);
    __syncthreads();
    const int ds = first_varying_digit(((ull)S.d3[0] << 32) | S.d3[1], S.d3[2], d0, ks.ndig);
    if (ds >= ks.ndig) {
        // All keys equal: the input order is the answer.
#pragma unroll
        for (int k = 0; k < kFinItems; k++) {
            uint32_t idx = warp * (kFinItems * 32) + k * 32 + lane;
            if (idx < c) emit(out_base + r0 + idx, v[k]);
        }
        return;
    }
    // Stable counting pass on digit ds (ranks as in k_pass).
#pragma unroll
    for (int k = 0; k < kFinItems; k++) {
        uint32_t idx = warp * (kFinItems * 32) + k * 32 + lane;
        dg[k] = idx < c ? digit_of(v[k], ds) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, dg[k]);
        uint32_t cnt = dg[k] < 256u ? S.wcnt[warp][dg[k]] : 0u;
        rk[k] = cnt + __popc(peers & lt_mask);
        __syncwarp();
        if (dg[k] < 256u && lane == __ffs(peers) - 1)
            S.wcnt[warp][dg[k]] = (uint16_t)(cnt + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    {
        const int dig = tid;
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kFinThreads / 32; ww++) {
            uint32_t cc = S.wcnt[ww][dig];
            S.wcnt[ww][dig] = (uint16_t)run;
            run += cc;
        }
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) S.warp_tot[warp] = incl;
        __syncthreads();
        uint32_t wp = 0;
#pragma unroll
        for (int ww = 0; ww < kFinThreads / 32; ww++) wp += ww < warp ? S.warp_tot[ww] : 0u;
        S.sb_off[dig] = (uint16_t)(wp + incl - run);
        S.sb_cnt[dig] = (uint16_t)run;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kFinItems; k++)
        if (dg[k] < 256u) B[r0 + S.sb_off[dg[k]] + S.wcnt[warp][dg[k]] + rk[k]] = v[k];
    __syncthreads();
    // Tiny sub-buckets: rank by comparison (ComparisonSort of Algorithm 1).
    for (uint32_t i = tid; i < c; i += kFinThreads) {
        const uint4 tv = B[r0 + i];
        const uint32_t dd = digit_of(tv, ds);
        const uint32_t so = S.sb_off[dd], sc = S.sb_cnt[dd];
        if (sc <= (uint32_t)kTiny) {
            uint32_t r = 0;
            for (uint32_t j = 0; j < sc; j++) r += tup_less(B[r0 + so + j], tv, ks.lo_mask) ? 1u : 0u;
            emit(out_base + r0 + so + r, tv);
        } else if (i == so) {
            int slot = atomicAdd(&S.stk_n, 1);
            if (slot < kFinStack) {
                S.stk_s[slot] = r0 + so;
                S.stk_c[slot] = sc;
            } else {
                atomicOr(err, kErrCapacity);
            }
        }
    }
    // caller synchronises before reading the stack
    (void)ds;
}

template <int MODE>
__global__ void __launch_bounds__(kFinThreads)
k_finish(Work w, KeySpec ks, Emitter<MODE> emit) {
    extern __shared__ uint4 B[];  // kSmall tuples
    __shared__ FinShared S;
    const ull nfin = w.ctl->fin_count < w.cap_fin ? w.ctl->fin_count : w.cap_fin;
    const int tid = threadIdx.x;
    while (true) {
        __syncthreads();
        if (tid == 0) {
            S.task = atomicAdd(&w.ctl->fin_ctr, 1u);
            S.stk_n = 0;
        }
        __syncthreads();
        const uint32_t ti = S.task;
        if (ti >= nfin) break;
        const FinTask tk = w.fin[ti];
        const uint4* src = w.tup[tk.buf] + tk.start;
        if (tk.flags & 1) {  // all keys equal: input order
            for (uint32_t i = tid; i < tk.count; i += kFinThreads) emit(tk.start + i, src[i]);
            continue;
        }
        if (tk.count > (uint32_t)kSmall) {  // never produced by k_classify
            if (tid == 0) atomicOr(w.err, kErrCapacity);
            continue;
        }
        fin_range<MODE>(B, S, src, 0, tk.count, tk.digit, ks, emit, tk.start, w.err);
        while (true) {
            __syncthreads();
            const int ns = S.stk_n;
            if (ns <= 0) break;
            const int top = (ns > kFinStack ? kFinStack : ns) - 1;
            const uint32_t s0 = S.stk_s[top], c0 = S.stk_c[top];
            __syncthreads();
            if (tid == 0) S.stk_n = top;
            // digit: the sub-bucket's first digit is shared, so restarting at
            // 0 only costs the difference scan; keys decide.
            fin_range<MODE>(B, S, nullptr, s0, c0, 0, ks, emit, tk.start, w.err);
        }
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

cudaError_t launch_extract_records(const LaunchCfg& c, const uint8_t* in, ull n, uint32_t rec,
                                   KeySpec ks, const Work& w, int hist_digit) {
    if (rec == 100)
        k_extract_records<100><<<c.grid, 256, 0, c.stream>>>(in, n, rec, ks, w.tup[0], w.hist[0],
                                                             w.diff[0], hist_digit);
    else
        k_extract_records<0><<<c.grid, 256, 0, c.stream>>>(in, n, rec, ks, w.tup[0], w.hist[0],
                                                           w.diff[0], hist_digit);
    return cudaGetLastError();
}

cudaError_t launch_extract_pairs(const LaunchCfg& c, const uint64_t* keys, const uint32_t* idx,
                                 ull n, KeySpec, const Work& w) {
    k_extract_pairs<<<c.grid, 256, 0, c.stream>>>(keys, idx, n, w.tup[0], w.hist[0], w.diff[0]);
    return cudaGetLastError();
}

cudaError_t launch_init(cudaStream_t s, const Work& w, ull n, int digit0) {
    k_init<<<1, 32, 0, s>>>(w, n, digit0);
    return cudaGetLastError();
}

cudaError_t launch_hist(const LaunchCfg& c, const Work& w, KeySpec ks, int level) {
    k_hist<<<c.grid, kPassThreads, 0, c.stream>>>(w, ks, level);
    return cudaGetLastError();
}

cudaError_t launch_classify(const LaunchCfg& c, const Work& w, KeySpec ks, int level) {
    k_classify<<<c.grid, 128, 0, c.stream>>>(w, ks, level);
    return cudaGetLastError();
}

cudaError_t launch_classify_partition(cudaStream_t s, const Work& w) {
    k_classify_partition<<<1, 32, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_pass(const LaunchCfg& c, const Work& w, KeySpec ks, int level) {
    k_pass<<<c.grid, kPassThreads, c.smem, c.stream>>>(w, ks, level);
    return cudaGetLastError();
}

cudaError_t launch_finish_records(const LaunchCfg& c, const Work& w, KeySpec ks) {
    Emitter<0> e;
    e.perm = w.perm;
    k_finish<0><<<c.grid, kFinThreads, c.smem, c.stream>>>(w, ks, e);
    return cudaGetLastError();
}

cudaError_t launch_finish_pairs(const LaunchCfg& c, const Work& w, KeySpec ks, uint64_t* keys_out,
                                uint32_t* idx_out) {
    Emitter<1> e;
    e.keys = keys_out;
    e.idx = idx_out;
    k_finish<1><<<c.grid, kFinThreads, c.smem, c.stream>>>(w, ks, e);
    return cudaGetLastError();
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
        case KK_FINISH_PAIRS: return (size_t)kSmall * sizeof(uint4);
        default: return 0;
    }
}

int kernel_threads(KernelKind k) {
    switch (k) {
        case KK_PASS:
        case KK_HIST: return kPassThreads;
        case KK_FINISH_REC:
        case KK_FINISH_PAIRS: return kFinThreads;
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
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_extract_records<100>, 256, 0);
        g_bps[KK_EXTRACT_REC] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_extract_pairs, 256, 0);
        g_bps[KK_EXTRACT_PAIRS] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_hist, kPassThreads, 0);
        g_bps[KK_HIST] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_pass, kPassThreads,
                                                      kernel_smem(KK_PASS));
        g_bps[KK_PASS] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_finish<0>, kFinThreads,
                                                      kernel_smem(KK_FINISH_REC));
        g_bps[KK_FINISH_REC] = v > 0 ? v : 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_finish<1>, kFinThreads,
                                                      kernel_smem(KK_FINISH_PAIRS));
        g_bps[KK_FINISH_PAIRS] = v > 0 ? v : 1;
        g_bps[KK_GATHER100] = gather_blocks_per_sm(KK_GATHER100);
        g_bps[KK_GATHER100_TMA] = gather_blocks_per_sm(KK_GATHER100_TMA);
        g_bps[KK_GATHER_GENERIC] = gather_blocks_per_sm(KK_GATHER_GENERIC);
        g_bps_init = true;
    }
    return g_bps[k];
}

}  // namespace ley
