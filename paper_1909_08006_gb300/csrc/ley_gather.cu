// Record gather: out[j] = in[perm[j]] -- the record scatter of Section 3.2
// ("scatter data records ... given the sorted (key, pointer) tuples"), done on
// the GPU as a gather so that the output is written sequentially.
//
// A 100-byte record starts at byte 100*i, which is only 4-byte aligned
// (100 mod 16 = 4).  Both gather kernels fetch the 16-byte aligned 112-byte
// window [floor(100 i / 16) * 16, +112) that holds it (always the same four
// 32-byte sectors), shift it by 0..3 words and stage 32 records = 3200
// contiguous output bytes per warp in shared memory, then write the tile with
// 16-byte stores (LSU kernel) or one TMA bulk store (TMA kernel).  No access
// leaves a 16-byte granule that holds record bytes.
#define LEY_FILE_ID 2
#include "ley_kernels.h"
#include "ley_rec100.cuh"
#include "ley_tma.cuh"

namespace ley {

using ull = unsigned long long;

constexpr int kChunk = 32;                     // records per warp tile
constexpr int kChunkBytes = kChunk * kRec;     // 3200

__device__ __forceinline__ uint4 ldg_nc_na(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// --------------------------------------------------------------- LSU path

constexpr int kGatherWarps = 8;

__global__ void __launch_bounds__(kGatherWarps * 32)
k_gather100(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
            const uint32_t* __restrict__ perm, ull n, ull n_in, uint32_t* err) {
    __shared__ __align__(16) uint32_t stage[kGatherWarps][kChunk * kRecWords];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ull nchunks = (n + kChunk - 1) / kChunk;
    uint32_t* st = stage[warp];
    for (ull c = (ull)blockIdx.x * kGatherWarps + warp; c < nchunks;
         c += (ull)gridDim.x * kGatherWarps) {
        const ull j = c * kChunk + lane;
        const bool valid = j < n;
        uint32_t w[28];
        uint32_t o = 0;
        if (valid) {
            uint32_t pj = __ldg(perm + j);
            if (pj >= n_in) {  // never for a valid permutation; keeps reads in bounds
                LEY_FAIL(err, kErrCapacity);
                pj = 0;
            }
            const ull s = (ull)pj * kRec;
            const uint4* p = reinterpret_cast<const uint4*>(in + (s & ~15ull));
            o = (uint32_t)(s & 15) >> 2;
#pragma unroll
            for (int q = 0; q < 7; q++) {
                uint4 v = ldg_nc_na(p + q);
                w[4 * q] = v.x;
                w[4 * q + 1] = v.y;
                w[4 * q + 2] = v.z;
                w[4 * q + 3] = v.w;
            }
            shift_store(st + lane * kRecWords, w, o);
        }
        __syncwarp();
        uint8_t* dst = out + c * kChunkBytes;
        const ull nvalid = n - c * kChunk < (ull)kChunk ? n - c * kChunk : (ull)kChunk;
        if (nvalid == kChunk) {
            const uint4* s4 = reinterpret_cast<const uint4*>(st);
            uint4* d4 = reinterpret_cast<uint4*>(dst);
            for (int q = lane; q < kChunkBytes / 16; q += 32) __stcs(d4 + q, s4[q]);
        } else {
            uint32_t* d1 = reinterpret_cast<uint32_t*>(dst);
            for (int q = lane; q < (int)nvalid * kRecWords; q += 32) d1[q] = st[q];
        }
        __syncwarp();
    }
}

// --------------------------------------------------------------- TMA path

constexpr int kTmaWarps = 4;
constexpr int kTmaBufs = 2;

struct __align__(128) TmaWarpBuf {
    uint8_t win[kTmaBufs][kChunk * kWinBytes];     // 2 x 3584
    uint32_t stage[kTmaBufs][kChunk * kRecWords];  // 2 x 3200
};

// Issue the window loads of chunk c into buffer b; returns this lane's word
// offset (record start within its window).
__device__ __forceinline__ uint32_t tma_issue(TmaWarpBuf& wb, uint64_t* bar, int b, ull c,
                                              const uint8_t* in, const uint32_t* perm, ull n,
                                              ull n_in, int lane, uint32_t* err) {
    const ull j = c * kChunk + lane;
    const ull nvalid = n - c * kChunk < (ull)kChunk ? n - c * kChunk : (ull)kChunk;
    uint32_t o = 0;
    const uint8_t* src = nullptr;
    if (j < n) {
        uint32_t pj = __ldg(perm + j);
        if (pj >= n_in) {  // never for a valid permutation; keeps reads in bounds
            LEY_FAIL(err, kErrCapacity);
            pj = 0;
        }
        const ull s = (ull)pj * kRec;
        src = in + (s & ~15ull);
        o = (uint32_t)(s & 15) >> 2;
    }
    if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)nvalid * kWinBytes);
    __syncwarp();
    if (j < n) tma_load_1d(wb.win[b] + lane * kWinBytes, src, kWinBytes, bar);
    return o;
}

__global__ void __launch_bounds__(kTmaWarps * 32)
k_gather100_tma(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                const uint32_t* __restrict__ perm, ull n, ull n_in, uint32_t* err) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    TmaWarpBuf* bufs = reinterpret_cast<TmaWarpBuf*>(smem_raw);
    __shared__ __align__(8) uint64_t bars[kTmaWarps][kTmaBufs];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    TmaWarpBuf& wb = bufs[warp];
    if (lane == 0) {
        for (int b = 0; b < kTmaBufs; b++) mbar_init(&bars[warp][b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const ull nchunks = (n + kChunk - 1) / kChunk;
    const ull first = (ull)blockIdx.x * kTmaWarps + warp;
    const ull stride = (ull)gridDim.x * kTmaWarps;
    uint32_t o[kTmaBufs] = {0, 0};
    uint32_t phase[kTmaBufs] = {0, 0};
    bool ok = true;
    for (int b = 0; b < kTmaBufs; b++) {
        ull c = first + b * stride;
        if (c < nchunks) o[b] = tma_issue(wb, &bars[warp][b], b, c, in, perm, n, n_in, lane, err);
    }
    int it = 0;
    for (ull c = first; c < nchunks; c += stride, it++) {
        const int b = it & 1;
        if (!mbar_wait(&bars[warp][b], phase[b])) {
            ok = false;
            break;
        }
        phase[b] ^= 1;
        // The bulk store that last read stage[b] must be done reading it.
        if (lane == 0) bulk_wait_read_1();
        __syncwarp();
        const ull nvalid = n - c * kChunk < (ull)kChunk ? n - c * kChunk : (ull)kChunk;
        if ((ull)lane < nvalid) {
            const uint4* win4 = reinterpret_cast<const uint4*>(wb.win[b] + lane * kWinBytes);
            uint32_t w[28];
#pragma unroll
            for (int q = 0; q < 7; q++) {
                uint4 v = win4[q];
                w[4 * q] = v.x;
                w[4 * q + 1] = v.y;
                w[4 * q + 2] = v.z;
                w[4 * q + 3] = v.w;
            }
            shift_store(wb.stage[b] + lane * kRecWords, w, o[b]);
        }
        __syncwarp();
        uint8_t* dst = out + c * kChunkBytes;
        if (nvalid == kChunk) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                tma_store_1d(dst, wb.stage[b], kChunkBytes);
                bulk_commit();
            }
        } else {
            uint32_t* d1 = reinterpret_cast<uint32_t*>(dst);
            for (int q = lane; q < (int)nvalid * kRecWords; q += 32) d1[q] = wb.stage[b][q];
        }
        __syncwarp();
        // Window b is consumed: refill it with chunk c + 2*stride.
        const ull cn = c + kTmaBufs * stride;
        if (cn < nchunks) o[b] = tma_issue(wb, &bars[warp][b], b, cn, in, perm, n, n_in, lane, err);
    }
    if (!ok) {
        if (lane == 0) LEY_FAIL(err, kErrTimeout);
        // Give copies still in flight a bounded chance to land before exit.
        for (int b = 0; b < kTmaBufs; b++) (void)mbar_wait(&bars[warp][b], phase[b]);
    }
    if (lane == 0) bulk_wait_read_0();
    __syncwarp();
}

// ------------------------------------------------------------ generic path

// Any rec_bytes.  A multiple of 4 is copied in words, one warp per record.
// Other sizes are copied byte by byte, one warp per 32 consecutive output
// records: lane l loads the source index of record l of the group, and the
// warp writes the group's cnt * rec output bytes contiguously, each lane
// taking the source index of its byte's record from the lane that loaded it.
__global__ void __launch_bounds__(256)
k_gather_generic(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                 const uint32_t* __restrict__ perm, ull n, ull n_in, uint32_t rec) {
    const int lane = threadIdx.x & 31;
    const ull warps = (ull)gridDim.x * (blockDim.x >> 5);
    const ull warp0 = (ull)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if ((rec & 3u) == 0) {
        const uint32_t words = rec / 4;
        for (ull j = warp0; j < n; j += warps) {
            uint32_t pj = __ldg(perm + j);
            if (pj >= n_in) pj = 0;  // never for a valid permutation; keeps reads in bounds
            const uint32_t* s = reinterpret_cast<const uint32_t*>(in + (ull)pj * rec);
            uint32_t* d = reinterpret_cast<uint32_t*>(out + j * rec);
            for (uint32_t q = lane; q < words; q += 32) d[q] = __ldg(s + q);
        }
        return;
    }
    const ull groups = (n + 31) / 32;
    for (ull g = warp0; g < groups; g += warps) {
        const ull j0 = g * 32;
        const uint32_t cnt = (uint32_t)min((ull)32, n - j0);
        uint32_t pj = (uint32_t)lane < cnt ? __ldg(perm + j0 + lane) : 0u;
        if (pj >= n_in) pj = 0;  // never for a valid permutation; keeps reads in bounds
        const uint32_t bytes = cnt * rec;
        uint8_t* d = out + j0 * rec;
        for (uint32_t b0 = 0; b0 < bytes; b0 += 32) {  // the same trip count on every lane
            const uint32_t b = b0 + (uint32_t)lane;
            const uint32_t r = min(b / rec, cnt - 1);
            const uint32_t p = __shfl_sync(0xffffffffu, pj, (int)r);
            if (b < bytes) d[b] = __ldg(in + (ull)p * rec + (b - r * rec));
        }
    }
}

// ------------------------------------------------------- wait self-test
//
// Failure detection without a GPU fault: one of the library's bounded waits
// is made to give up on purpose, against a condition that nothing will ever
// satisfy -- a device word nobody writes (the scan look-back's kind of wait)
// or an mbarrier whose transaction bytes no copy delivers (the TMA gathers'
// kind) -- and must latch kErrTimeout and return, leaving the context usable.
__global__ void k_selftest_wait(uint32_t which, const unsigned long long* never_set,
                                uint32_t* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (which == 0) {
        uint32_t spins = 0;
        while (*(volatile const unsigned long long*)never_set == 0) {
            if (++spins > kSpinLimit) {
                LEY_FAIL(err, kErrTimeout);
                break;
            }
            if (spins > 32) __nanosleep(64);
        }
    } else {
        mbar_init(&bar, 1);
        mbar_fence_init();
        mbar_arrive_expect_tx(&bar, 16);  // 16 bytes that never arrive
        if (!mbar_wait(&bar, 0)) LEY_FAIL(err, kErrTimeout);
    }
}

cudaError_t launch_selftest_wait(cudaStream_t s, uint32_t which,
                                 const unsigned long long* never_set, uint32_t* err) {
    k_selftest_wait<<<1, 32, 0, s>>>(which, never_set, err);
    return cudaGetLastError();
}

// -------------------------------------------------------------- launchers

static size_t tma_smem() { return (size_t)kTmaWarps * sizeof(TmaWarpBuf); }

int gather_blocks_per_sm(KernelKind k) {
    int v = 0;
    if (k == KK_GATHER100) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_gather100, kGatherWarps * 32, 0);
    } else if (k == KK_GATHER100_TMA) {
        cudaFuncSetAttribute(k_gather100_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tma_smem());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_gather100_tma, kTmaWarps * 32,
                                                      tma_smem());
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_gather_generic, 256, 0);
    }
    return v > 0 ? v : 1;
}

extern uint32_t* device_err_word();
cudaError_t launch_gather_err(const LaunchCfg& c, const uint8_t* in, uint8_t* out,
                              const uint32_t* perm, ull n, ull n_in, uint32_t rec, int variant,
                              uint32_t* err);

cudaError_t launch_gather(const LaunchCfg& c, const uint8_t* in, uint8_t* out,
                          const uint32_t* perm, ull n, ull n_in, uint32_t rec, int variant) {
    return launch_gather_err(c, in, out, perm, n, n_in, rec, variant, device_err_word());
}

// Same kernels as launch_gather, with the device status word given by the
// caller instead of the library's per-device word.
cudaError_t launch_gather_err(const LaunchCfg& c, const uint8_t* in, uint8_t* out,
                              const uint32_t* perm, ull n, ull n_in, uint32_t rec, int variant,
                              uint32_t* err) {
    if (rec == kRec && variant == 1) {
        k_gather100_tma<<<c.grid, kTmaWarps * 32, tma_smem(), c.stream>>>(in, out, perm, n, n_in,
                                                                          err);
    } else if (rec == kRec) {
        k_gather100<<<c.grid, kGatherWarps * 32, 0, c.stream>>>(in, out, perm, n, n_in, err);
    } else {
        k_gather_generic<<<c.grid, 256, 0, c.stream>>>(in, out, perm, n, n_in, rec);
    }
    return cudaGetLastError();
}

}  // namespace ley
