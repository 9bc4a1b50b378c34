// Shared definitions of the leysort CUDA library (device and host side).
//
// Sorting works on 16-byte (key, pointer) tuples, the representation of
// Section 3.2 ("Leyenda extracts the (key, pointer) tuples from records"):
//   x = key bytes 4..7   (big-endian: byte 4 in bits 31..24)
//   y = key bytes 0..3   (big-endian)
//   z = key bytes 8..11  (big-endian) -- or, for key/payload pairs, the payload
//   w = input index (the pointer)
// so that (y, x) read as one u64 is key bytes 0..7 as a big-endian integer and
// comparing (y:x, z, w) as unsigned integers is the stable key order.  Bytes
// past key_bytes are stored as zero.  Digit d of Algorithm 1 is key byte d.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ley {

constexpr int kRadix = 256;
constexpr int kMaxDigits = 12;      // key bytes a tuple can hold
constexpr int kMaxLevels = 12;      // one MSD level per digit at most

// Tile of the multi-CTA passes (histogram and scatter): 4096 tuples.  The
// scatter pass uses 512 threads x 8 items, the histogram 256 threads x 16.
constexpr int kPassTile = 4096;
constexpr int kPassThreads = 512;
constexpr int kPassItems = kPassTile / kPassThreads;   // 8
constexpr int kPassWarps = kPassThreads / 32;          // 16
constexpr int kHistThreads = 512;
constexpr int kHistItems = kPassTile / kHistThreads;   // 8
// Tiles per chunk of the per-tile offset scan.
constexpr int kScanChunk = 16;
constexpr uint32_t kNoPass = 0xFFFFFFFFu;

// In-CTA finishing (the small-bucket queue of Algorithm 1): 256 threads x 8.
constexpr int kFinThreads = 256;
constexpr int kFinWarps = kFinThreads / 32;
constexpr int kFinItems = 8;
constexpr int kSmall = kFinThreads * kFinItems;        // 2048 tuples: big-bucket threshold
constexpr int kTiny = 32;                              // tiny-bucket threshold (comparison rank)
constexpr int kWarpMax = 32 * kFinItems;               // sub-buckets one warp sorts (256)
constexpr uint32_t kFlagPiece = 8 * kSmall;              // pieces of an all-equal run (16384)
// Sub-buckets above kTiny inside one task are disjoint at each digit depth,
// so at most kSmall / (kTiny + 1) per depth and kMaxDigits depths: the
// queue never needs more slots than this and never wraps.
constexpr int kFinQueue = (kSmall / (kTiny + 1)) * 12 + 8;   // 752
constexpr int kFinStack = kSmall / (kWarpMax + 1) + 2;       // block stack (> kWarpMax)

// Device-side error bits (latched in the per-device status word).
constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrCapacity = 2u;

// Latches an error bit in the per-device status word and, for the first
// error only, where it was raised: (source file id << 16) | line.
__device__ __forceinline__ void ley_fail(uint32_t* err, uint32_t code, uint32_t site) {
    atomicOr(err, code);
    atomicCAS(err + 1, 0u, site);
}
#ifndef LEY_FILE_ID
#define LEY_FILE_ID 0
#endif
#define LEY_FAIL(err, code) ::ley::ley_fail((err), (code), (LEY_FILE_ID << 16) | __LINE__)

// Bounded waits: polls before a wait gives up (with nanosleep backoff this is
// well under a second on a healthy GPU, and terminates on a broken one).
constexpr uint32_t kSpinLimit = 1u << 22;

// One MSD segment: a bucket that still needs a multi-CTA pass.
struct __align__(16) Seg {
    unsigned long long start;
    uint32_t count;
    uint16_t digit;
    uint8_t buf;      // which tuple buffer holds it (0 or 1)
    uint8_t pad;
};

// One finishing task: a contiguous range of tuples, sorted in one CTA.
// flags bit 0: all keys in the range are equal (emit in place, any size).
struct __align__(16) FinTask {
    unsigned long long start;
    uint32_t count;
    uint16_t digit;
    uint8_t buf;
    uint8_t flags;
};

// Bits of the key that differ inside a segment (OR over tuples of t ^ ref).
struct __align__(16) Diff {
    unsigned long long hi;   // key bytes 0..7 (y:x)
    uint32_t lo;             // key bytes 8..11 (z, masked)
    uint32_t pad;
};

struct LevelCtl {
    unsigned long long big_packed;   // (#segments << 40) | #tiles of list L
    unsigned long long pass_count;   // buckets scattered at level L
    uint32_t scan_chunk_ctr;
    uint32_t pad[3];
};

struct Ctl {
    LevelCtl lvl[kMaxLevels + 1];
    unsigned long long fin_count;
    uint32_t fin_ctr;
    uint32_t gather_ctr;
    uint32_t pad[4];
};

constexpr int kPackShift = 40;
constexpr unsigned long long kPackMask = (1ull << kPackShift) - 1;

// Key description shared by all kernels of one sort.
struct KeySpec {
    int ndig;             // number of key bytes (digits)
    unsigned long long hi_mask;  // key bits of (y:x)
    uint32_t lo_mask;     // key bits of z (0 for key/payload pairs)
    uint32_t big;         // buckets above this many tuples are scattered again (<= kSmall)
    uint32_t tiny;        // sub-buckets up to this many are ranked by comparison (kTiny..kWarpMax)
};

// Device views of the scratch workspace of one internal sort.
struct Work {
    uint4* tup[2];
    uint32_t* perm;               // records mode: output permutation
    Ctl* ctl;
    Seg* segs[2];                 // big list per level parity
    uint32_t* seg_tile_base[2];
    uint32_t* seg_tile_owner[2];  // tile -> slot in the big list
    uint32_t* seg_pass[2];        // slot -> bucket_base row, or kNoPass
    uint32_t* hist[2];            // [cap_seg][256] bucket sizes
    Diff* diff[2];
    uint32_t* tile_cnt;           // [cap_tiles][256] digit counts, then offsets
    uint32_t* bucket_base;        // [cap_seg][256] exclusive offsets
    FinTask* fin;
    unsigned long long* status;   // [cap_chunks][256] scan look-back words
    uint32_t* err;                // per-device status word
    unsigned long long cap_seg, cap_fin, cap_tiles, cap_chunks;
    unsigned long long n;
};

// One request of a batched sort.  Requests lie back to back in the batch's
// tuple space, each starting on a tile boundary: request r owns tuple
// positions [off, off + n), and its tuples carry indices local to it.
struct BatchReq {
    const uint8_t* in;       // records, or u64 keys
    uint8_t* out;            // records, or u64 keys
    const uint32_t* idx_in;  // pairs: payloads
    uint32_t* idx_out;
    unsigned long long n;
    unsigned long long off;  // multiple of kPassTile
};

__host__ __device__ inline uint32_t ceil_div_u64(unsigned long long a, unsigned long long b) {
    return (uint32_t)((a + b - 1) / b);
}

}  // namespace ley
