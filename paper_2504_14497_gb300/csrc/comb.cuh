// Fixed-base comb tables (Section 2.4: encryption multiplies the fixed
// points G and H by random scalars; decryption checks candidate messages
// against multiples of G).  The table of a point X has 32 windows of 8
// bits; entry (window i, value v) is (v 2^(8i)) X, stored affine and
// quad-planar with stride COMB_POINTS (entries with v = 0 are unused).
#pragma once
#include <stdint.h>

#include "ec.cuh"

namespace pcmm {

constexpr int COMB_WINDOWS = 32;    // 8-bit windows of a 256-bit scalar
constexpr int COMB_ENTRIES = 256;   // v = 0..255 per window
constexpr int COMB_POINTS = COMB_WINDOWS * COMB_ENTRIES;

// R <- s X for s < 2^(8 nwin), from the comb table of X: one mixed
// addition per non-zero byte of s.
__device__ __forceinline__ void comb_mul_u64(jac& R, const uint4* __restrict__ tab, uint64_t s, int nwin) {
    jac_set_inf(R);
    aff T;
    for (int win = 0; win < nwin; win++) {
        const uint32_t v = (uint32_t)(s >> (8 * win)) & 0xffu;
        if (v) {
            load_aff(T, tab, COMB_POINTS, (size_t)win * COMB_ENTRIES + v);
            jac_madd(R, T);
        }
    }
}

// Device address of the generator's comb table on the current device, or
// nullptr when pcmm_init has not built it there.
const uint4* comb_table_G();

}  // namespace pcmm
