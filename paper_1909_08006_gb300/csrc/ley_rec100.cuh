// 100-byte records (the geometry of Section 4.1) in 16-byte granules.
//
// Record i starts at byte 100*i, which is only 4-byte aligned (100 mod 16 =
// 4).  The 16-byte aligned 112-byte window [floor(100 i / 16) * 16, +112)
// holds the whole record, always in the same four 32-byte sectors, and no
// 16-byte granule of it lies outside the record's own granules; the record
// begins 0..3 words into its window.
#pragma once

#include <cstdint>

namespace ley {

constexpr int kRec = 100;
constexpr int kRecWords = kRec / 4;            // 25
constexpr int kWinBytes = 112;                 // 7 x 16 B

// Copy words o..o+24 of a 28-word window into the staging tile.
__device__ __forceinline__ void shift_store(uint32_t* st, const uint32_t (&w)[28], uint32_t o) {
    switch (o) {
        case 0:
#pragma unroll
            for (int k = 0; k < kRecWords; k++) st[k] = w[k];
            break;
        case 1:
#pragma unroll
            for (int k = 0; k < kRecWords; k++) st[k] = w[k + 1];
            break;
        case 2:
#pragma unroll
            for (int k = 0; k < kRecWords; k++) st[k] = w[k + 2];
            break;
        default:
#pragma unroll
            for (int k = 0; k < kRecWords; k++) st[k] = w[k + 3];
            break;
    }
}

}  // namespace ley
