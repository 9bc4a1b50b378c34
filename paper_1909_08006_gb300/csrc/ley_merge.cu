// K-way merge of sorted runs (the merge stage of Section 3.2: the runs are
// merged into a globally sorted partition by a K-way merge), done on the GPU
// over 16-byte tuples by merge path (Green, McColl and Bader, "GPU Merge
// Path", 2012), generalised to k runs in one pass (below); a fan-in above
// kKwayMaxRuns is first brought down by rounds of pairwise merges.
//
// The k runs lie back to back in one tuple array, run r at [off[r], off[r+1]),
// each sorted by (key, position).  Positions grow with the run number, so
// comparing full tuples (key, then position) merges stably: on equal keys the
// lower run comes first, which is the order of the input.  In a pairwise
// round runs 2i and 2i+1 are merged into the other buffer at the same place
// (an odd last run is copied).
#define LEY_FILE_ID 3
#include "ley_kernels.h"

#include <cstring>

namespace ley {

using ull = unsigned long long;

constexpr int kMergeThreads = 256;
constexpr int kMergeItems = 4;
constexpr int kMergeTile = kMergeThreads * kMergeItems;   // 1024 outputs per tile

__device__ __forceinline__ bool mtup_less(const uint4& a, const uint4& b, uint32_t lo_mask) {
    const ull ka = ((ull)a.y << 32) | a.x, kb = ((ull)b.y << 32) | b.x;
    if (ka != kb) return ka < kb;
    const uint32_t la = a.z & lo_mask, lb = b.z & lo_mask;
    if (la != lb) return la < lb;
    return a.w < b.w;
}

// Number of A elements among the first d outputs of the stable merge of
// A[0, na) and B[0, nb) (A first on ties): the merge-path split of diagonal d.
template <class GetA, class GetB>
__device__ __forceinline__ uint32_t merge_split(uint32_t d, uint32_t na, uint32_t nb,
                                                GetA geta, GetB getb, uint32_t lo_mask) {
    uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        // A[mid] is among the first d outputs iff it precedes B[d - 1 - mid]
        if (mtup_less(geta(mid), getb(d - 1 - mid), lo_mask)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One merge round.  pair p merges runs 2p and 2p+1 of `off` (k runs); its
// output [off[2p], off[min(2p+2, k)]) is cut into tiles of kMergeTile, and
// the tiles of all pairs are numbered consecutively.
__global__ void __launch_bounds__(kMergeThreads)
k_merge_round(const uint4* __restrict__ src, uint4* __restrict__ dst, const ull* __restrict__ off,
              uint32_t k, uint32_t lo_mask) {
    __shared__ uint4 sa[kMergeTile];
    __shared__ uint4 so[kMergeTile];
    __shared__ uint32_t tile_base[65];
    const uint32_t npairs = (k + 1) / 2;
    if (threadIdx.x == 0) {
        uint32_t tb = 0;
        for (uint32_t p = 0; p < npairs && p < 64; p++) {
            tile_base[p] = tb;
            const ull len = off[min(2 * p + 2, k)] - off[2 * p];
            tb += (uint32_t)((len + kMergeTile - 1) / kMergeTile);
        }
        tile_base[min(npairs, 64u)] = tb;
    }
    __syncthreads();
    const uint32_t ntiles = tile_base[min(npairs, 64u)];
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint32_t p = 0;
        while (p + 1 < npairs && tile_base[p + 1] <= t) p++;
        const ull a0 = off[2 * p];
        const ull a1 = off[min(2 * p + 1, k)];
        const ull b1 = off[min(2 * p + 2, k)];
        const uint32_t na = (uint32_t)(a1 - a0), nb = (uint32_t)(b1 - a1);
        const uint32_t d0 = (t - tile_base[p]) * kMergeTile;
        const uint32_t d1 = min(d0 + kMergeTile, na + nb);
        const uint4* A = src + a0;
        const uint4* Bv = src + a1;
        auto ga = [&](uint32_t i) { return A[i]; };
        auto gb = [&](uint32_t i) { return Bv[i]; };
        const uint32_t s0 = merge_split(d0, na, nb, ga, gb, lo_mask);
        const uint32_t s1 = merge_split(d1, na, nb, ga, gb, lo_mask);
        // stage A[s0, s1) then B[d0 - s0, d1 - s1) in shared memory
        const uint32_t ca = s1 - s0, cb = (d1 - s1) - (d0 - s0), m = ca + cb;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m; i += kMergeThreads)
            sa[i] = i < ca ? A[s0 + i] : Bv[d0 - s0 + (i - ca)];
        __syncthreads();
        // each thread merges kMergeItems consecutive outputs of the tile
        const uint32_t my0 = min(threadIdx.x * kMergeItems, m);
        const uint32_t my1 = min(my0 + kMergeItems, m);
        auto la = [&](uint32_t i) { return sa[i]; };
        auto lb = [&](uint32_t i) { return sa[ca + i]; };
        uint32_t ia = merge_split(my0, ca, cb, la, lb, lo_mask);
        uint32_t ib = my0 - ia;
        for (uint32_t o = my0; o < my1; o++) {
            bool take_a;
            if (ia >= ca) take_a = false;
            else if (ib >= cb) take_a = true;
            else take_a = !mtup_less(sa[ca + ib], sa[ia], lo_mask);
            so[o] = take_a ? sa[ia++] : sa[ca + ib++];
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m; i += kMergeThreads) dst[a0 + d0 + i] = so[i];
    }
}

// ------------------------------------------------------ k-way merge path
//
// One pass over all k runs (k <= kKwayMaxRuns) instead of ceil(log2 k)
// pairwise rounds.  Every s-th tuple of every run is a sample, with
// s = kKwayTile / k (at most 256).  For each sample x the split vector
// split_r(x) = #{y in run r : y < x} is found by k binary searches, and its
// rank among all samples, q(x) = sum_r ceil(split_r(x) / s), by the same
// numbers (the samples of run r below x are those at positions below
// split_r(x)); the vector goes to row q(x) of a table, which is therefore the
// samples' split vectors in merged order, with the runs' ends as the last
// row.  The merged output between two consecutive samples holds at most s
// tuples of the first sample's run and fewer than s of every other run (one
// more would be a sample in between), so at most kKwayTile tuples: one CTA
// merges each such tile in shared memory, every tuple's place in the tile
// being its index in its own run's piece plus its lower bounds in the other
// pieces, and the tile's first output position the sum of its first row.
constexpr int kKwayThreads = 256;

__device__ __forceinline__ uint32_t kw_lower_bound(const uint4* a, uint32_t n, const uint4& x,
                                                   uint32_t lo_mask) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (mtup_less(a[mid], x, lo_mask)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One warp per sample; lane r handles run r.  table has (S + 1) rows of k.
__global__ void __launch_bounds__(256)
k_kmerge_samples(const uint4* __restrict__ tup, const ull* __restrict__ off, uint32_t k,
                 uint32_t s, uint32_t lo_mask, uint32_t* __restrict__ table, ull table_rows,
                 uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const ull gw = ((ull)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const ull nw = ((ull)gridDim.x * blockDim.x) >> 5;
    const uint32_t r = (uint32_t)lane;
    const ull r0 = r < k ? off[r] : 0, r1 = r < k ? off[r + 1] : 0;
    const uint32_t nr = (uint32_t)(r1 - r0);
    const uint32_t cr = (nr + s - 1) / s;  // samples of run r
    uint32_t incl = cr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t cb = incl - cr;  // first sample id of run r
    const uint32_t S = __shfl_sync(0xffffffffu, incl, 31);
    if ((ull)S + 1 > table_rows) {  // the host sized the table: never
        if (gw == 0 && lane == 0) LEY_FAIL(err, kErrCapacity);
        return;
    }
    if (gw == 0 && r < k) table[(ull)S * k + r] = nr;  // the last row: every run's end
    for (ull sid = gw; sid < S; sid += nw) {
        // the run of this sample: the highest run whose first sample id is
        // <= sid (an empty run shares its id with the next run)
        const uint32_t in_lo = __ballot_sync(0xffffffffu, r < k && cb <= (uint32_t)sid);
        const int i = 31 - __clz(in_lo);
        const uint32_t cbi = __shfl_sync(0xffffffffu, cb, i);
        const ull offi = __shfl_sync(0xffffffffu, r0, i);
        const uint32_t pos = ((uint32_t)sid - cbi) * s;
        const uint4 x = tup[offi + pos];
        uint32_t split = 0;
        if (r < k) split = r == (uint32_t)i ? pos : kw_lower_bound(tup + r0, nr, x, lo_mask);
        const uint32_t q = __reduce_add_sync(0xffffffffu, r < k ? (split + s - 1) / s : 0u);
        if (q >= S) {  // the ranks of the samples are a permutation of [0, S): never
            if (lane == 0) LEY_FAIL(err, kErrCapacity);
            continue;
        }
        if (r < k) table[(ull)q * k + r] = split;
    }
}

// One CTA per tile of consecutive table rows; perm[j] = the w field (the
// position in the concatenated runs) of the j-th tuple of the merge.
__global__ void __launch_bounds__(kKwayThreads)
k_kmerge_tiles(const uint4* __restrict__ tup, const ull* __restrict__ off, uint32_t k,
               const uint32_t* __restrict__ table, uint32_t S, uint32_t lo_mask,
               uint32_t* __restrict__ perm, ull n, uint32_t* err) {
    extern __shared__ uint4 sm[];  // kKwayTile tuples
    __shared__ uint32_t t_lo[kKwayMaxRuns], pre[kKwayMaxRuns + 1];
    __shared__ ull t_base, run0[kKwayMaxRuns];
    const int tid = threadIdx.x;
    for (uint32_t q = blockIdx.x; q < S; q += gridDim.x) {
        __syncthreads();  // the previous tile's shared state is no longer read
        if (tid < (int)k) {
            const uint32_t a = table[(ull)q * k + tid], b = table[(ull)(q + 1) * k + tid];
            t_lo[tid] = a;
            pre[tid + 1] = b >= a ? b - a : 0u;
            run0[tid] = off[tid];
            if (b < a) LEY_FAIL(err, kErrCapacity);  // rows out of order: never
        }
        __syncthreads();
        if (tid == 0) {
            ull base = 0;
            pre[0] = 0;
            for (uint32_t r = 0; r < k; r++) {
                base += t_lo[r];
                pre[r + 1] += pre[r];
            }
            t_base = base;
        }
        __syncthreads();
        const uint32_t total = pre[k];
        const ull base = t_base;
        if (total > (uint32_t)kKwayTile || base + total > n) {  // never for a valid table
            if (tid == 0) LEY_FAIL(err, kErrCapacity);
            continue;
        }
        for (uint32_t f = tid; f < total; f += kKwayThreads) {
            uint32_t lo = 0, hi = k;  // the run whose piece holds f: pre[r] <= f < pre[r + 1]
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (pre[mid] <= f) lo = mid;
                else hi = mid;
            }
            sm[f] = tup[run0[lo] + t_lo[lo] + (f - pre[lo])];
        }
        __syncthreads();
        for (uint32_t f = tid; f < total; f += kKwayThreads) {
            uint32_t a = 0, hi = k;
            while (hi - a > 1) {
                const uint32_t mid = (a + hi) >> 1;
                if (pre[mid] <= f) a = mid;
                else hi = mid;
            }
            const uint4 e = sm[f];
            uint32_t rank = f - pre[a];
            for (uint32_t r = 0; r < k; r++)
                if (r != a) rank += kw_lower_bound(sm + pre[r], pre[r + 1] - pre[r], e, lo_mask);
            if (rank < total) perm[base + rank] = e.w;
            else LEY_FAIL(err, kErrCapacity);  // inconsistent order: never
        }
    }
}

uint32_t kway_sample_step(uint32_t k) {
    const uint32_t s = (uint32_t)kKwayTile / (k ? k : 1);
    return s > 256 ? 256 : s;
}

// One warp per sample and one CTA per tile, not persistent grids: in the
// external sort these kernels run beside the gathers that feed the copies to
// the host, and CTAs that end after one tile let those higher-priority
// gathers onto the SMs (measured at 4e8 records: output copied at 157-160
// GB/s each way against 145-149 with three persistent CTAs per SM, and the
// merge itself 2.5 ms per partition against 4.0).
cudaError_t launch_kmerge(cudaStream_t st, int sms, const uint4* tup, const ull* off_dev,
                          uint32_t k, uint32_t S, uint32_t lo_mask, uint32_t* table,
                          ull table_rows, uint32_t* perm, ull n, uint32_t* err) {
    (void)sms;
    const uint32_t s = kway_sample_step(k);
    const int sgrid = (int)(((ull)S * 32 + 255) / 256 + 1);
    k_kmerge_samples<<<sgrid, 256, 0, st>>>(tup, off_dev, k, s, lo_mask, table, table_rows, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || S == 0) return e;
    e = cudaFuncSetAttribute(k_kmerge_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kKwayTile * sizeof(uint4)));
    if (e != cudaSuccess) return e;
    const int tgrid = (int)S;
    k_kmerge_tiles<<<tgrid, kKwayThreads, kKwayTile * sizeof(uint4), st>>>(
        tup, off_dev, k, table, S, lo_mask, perm, n, err);
    return cudaGetLastError();
}

// ------------------------------------------------ partition planning
//
// The external sort's partition cuts (Section 3.2: the merge is cut into
// independent pieces) from the device: the co-rank of every candidate --
// record p of run i, at p = step - 1, 2 step - 1, ... -- in the merged order
// (key, run, position), i.e. for every run j the number of its records
// before the candidate: p in its own run, elsewhere a binary search for the
// records with a smaller key, or with a key no larger in a lower run.  One
// warp per candidate, lane j searching run j (run j + 32, ... for k > 32).
// Runs are in device memory or in pinned host memory mapped for the device
// (the searches then read a few sectors per probe over the host link).

// Key bytes kb (<= 12) of the record at r as (bytes 0..7, bytes 8..11), big
// endian, bytes past kb zero: the unsigned order of (hi, lo) is memcmp's.
// Only the 16-byte granules that hold key bytes are read.
__device__ __forceinline__ void plan_key(const uint8_t* r, uint32_t kb, ull* hi, uint32_t* lo) {
    const uintptr_t a = (uintptr_t)r;
    const uint4* p = reinterpret_cast<const uint4*>(a & ~(uintptr_t)15);
    const uint32_t o = (uint32_t)(a & 15);
    const uint4 c0 = p[0];
    const uint4 c1 = o + kb > 16 ? p[1] : make_uint4(0, 0, 0, 0);
    const uint32_t wv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    uint32_t b[12];
#pragma unroll
    for (int i = 0; i < 12; i++) {
        const uint32_t q = o + i;
        uint32_t word = wv[0];
#pragma unroll
        for (int w2 = 1; w2 < 8; w2++) word = (q >> 2) == (uint32_t)w2 ? wv[w2] : word;
        b[i] = (uint32_t)i < kb ? (word >> (8 * (q & 3))) & 0xFFu : 0u;
    }
    ull h = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) h = (h << 8) | b[i];
    *hi = h;
    *lo = (b[8] << 24) | (b[9] << 16) | (b[10] << 8) | b[11];
}

__global__ void __launch_bounds__(256)
k_corank(const PlanRun* __restrict__ runs, uint32_t k, uint32_t rec, uint32_t kb,
         const ull* __restrict__ cbase, ull step, uint32_t ncand, uint32_t* __restrict__ split,
         ull* __restrict__ rank, uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const ull gw = ((ull)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const ull nw = ((ull)gridDim.x * blockDim.x) >> 5;
    for (ull c = gw; c < ncand; c += nw) {
        // the candidate's run: the last run whose first candidate is <= c
        uint32_t lo = 0, hi = k;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (cbase[mid] <= c) lo = mid;
            else hi = mid;
        }
        const uint32_t i = lo;
        const ull p = (c - cbase[i] + 1) * step - 1;
        if (p >= runs[i].len) {  // the host counted the candidates: never
            if (lane == 0) LEY_FAIL(err, kErrCapacity);
            continue;
        }
        ull khi;
        uint32_t klo;
        plan_key(runs[i].base + p * rec, kb, &khi, &klo);
        ull sum = 0;
        for (uint32_t j = lane; j < k; j += 32) {
            ull x;
            if (j == i) {
                x = p;
            } else {
                const bool upper = j < i;  // equal keys of a lower run come first
                const uint8_t* b = runs[j].base;
                ull l = 0, h = runs[j].len;
                while (l < h) {
                    const ull mid = (l + h) >> 1;
                    ull mh;
                    uint32_t ml;
                    plan_key(b + mid * rec, kb, &mh, &ml);
                    const bool less = mh < khi || (mh == khi && ml < klo);
                    const bool eq = mh == khi && ml == klo;
                    if (less || (upper && eq)) l = mid + 1;
                    else h = mid;
                }
                x = l;
            }
            split[c * k + j] = (uint32_t)x;
            sum += x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) rank[c] = sum;
    }
}

cudaError_t launch_corank(cudaStream_t st, int sms, const PlanRun* runs, uint32_t k, uint32_t rec,
                          uint32_t kb, const ull* cbase, ull step, uint32_t ncand, uint32_t* split,
                          ull* rank, uint32_t* err) {
    if (ncand == 0) return cudaSuccess;
    const int grid = (int)min((ull)sms * 8, ((ull)ncand * 32 + 255) / 256);
    k_corank<<<grid, 256, 0, st>>>(runs, k, rec, kb, cbase, step, ncand, split, rank, err);
    return cudaGetLastError();
}

cudaError_t launch_merge_round(cudaStream_t s, int grid, const uint4* src, uint4* dst,
                               const ull* off_dev, uint32_t k, uint32_t lo_mask) {
    k_merge_round<<<grid, kMergeThreads, 0, s>>>(src, dst, off_dev, k, lo_mask);
    return cudaGetLastError();
}

// After a round over `runs` runs, the merged pairs are the next round's runs:
// off'[i] = off[min(2i, runs)] for i = 0 .. ceil(runs / 2).  In place: entry
// i is written after every read of entries < 2i.
__global__ void k_halve_offsets(ull* off, uint32_t runs) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint32_t np = (runs + 1) / 2;
    for (uint32_t i = 1; i <= np; i++) off[i] = off[min(2 * i, runs)];
}

cudaError_t launch_halve_offsets(cudaStream_t s, ull* off, uint32_t runs) {
    k_halve_offsets<<<1, 32, 0, s>>>(off, runs);
    return cudaGetLastError();
}

// Writes up to kMaxOffsets run offsets, passed by value in the kernel's
// parameters (so the host needs no pinned copy buffer), to dst.
struct OffsetBlock {
    ull v[kMaxOffsets];
};

__global__ void k_set_offsets(ull* dst, OffsetBlock b, uint32_t count) {
    for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) dst[i] = b.v[i];
}

cudaError_t launch_set_offsets(cudaStream_t s, ull* dst, const ull* host, uint32_t count) {
    if (count > (uint32_t)kMaxOffsets) return cudaErrorInvalidValue;
    OffsetBlock b;
    for (uint32_t i = 0; i < count; i++) b.v[i] = host[i];
    k_set_offsets<<<1, 128, 0, s>>>(dst, b, count);
    return cudaGetLastError();
}

// Host bytes to device memory through kernel parameters, 4 KB per launch.
constexpr int kUploadChunk = 4000;
struct UploadBlock {
    unsigned char b[kUploadChunk];
};

__global__ void k_upload(unsigned char* dst, UploadBlock blk, uint32_t bytes) {
    for (uint32_t i = threadIdx.x; i < bytes; i += blockDim.x) dst[i] = blk.b[i];
}

cudaError_t launch_upload(cudaStream_t s, void* dst, const void* src, size_t bytes) {
    const unsigned char* h = static_cast<const unsigned char*>(src);
    unsigned char* d = static_cast<unsigned char*>(dst);
    for (size_t o = 0; o < bytes; o += kUploadChunk) {
        const uint32_t m = (uint32_t)(bytes - o < (size_t)kUploadChunk ? bytes - o : kUploadChunk);
        UploadBlock blk;
        std::memcpy(blk.b, h + o, m);
        k_upload<<<1, 256, 0, s>>>(d + o, blk, m);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Uniform random bytes (SplitMix64 of the 8-byte word index and a seed), for
// tuning runs.
__global__ void k_fill_random(uint8_t* p, ull bytes, ull seed) {
    const ull words = bytes / 8;
    for (ull i = (ull)blockIdx.x * blockDim.x + threadIdx.x; i < (bytes + 7) / 8;
         i += (ull)gridDim.x * blockDim.x) {
        ull z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        if (i < words) {
            reinterpret_cast<ull*>(p)[i] = z;
        } else {
            for (ull b = i * 8; b < bytes; b++) p[b] = (uint8_t)(z >> (8 * (b - i * 8)));
        }
    }
}

cudaError_t launch_fill_random(cudaStream_t s, uint8_t* p, ull bytes, ull seed) {
    k_fill_random<<<1024, 256, 0, s>>>(p, bytes, seed);
    return cudaGetLastError();
}

// Copies the tuples' input positions (the w field) out as the permutation.
__global__ void k_tuple_index(const uint4* __restrict__ t, uint32_t* __restrict__ perm, ull n) {
    for (ull i = (ull)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (ull)gridDim.x * blockDim.x)
        perm[i] = t[i].w;
}

cudaError_t launch_tuple_index(cudaStream_t s, int grid, const uint4* t, uint32_t* perm, ull n) {
    k_tuple_index<<<grid, 256, 0, s>>>(t, perm, n);
    return cudaGetLastError();
}

}  // namespace ley
