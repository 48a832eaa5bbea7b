// Prime-field arithmetic in F_p for NIST P-256, p = 2^256 - 2^224 + 2^192 + 2^96 - 1
// (Section 4.1), on sm_103a.
//
// Representation: 8 x 32-bit little-endian limbs held in registers.  Values
// are kept WEAKLY reduced: any integer in [0, 2^256) that is congruent to the
// field element (so 0 may appear as 0 or as p).  fe_canon() gives the unique
// representative below p; it is applied only when a result leaves the
// library or when a value must be compared.
//
// Multiplication: 8x8-limb operand scanning, one row per limb of b.  Each
// limb product is a single 32x32->64-bit multiply-add (mad.wide.u32, which
// also adds the row's running word), and the high halves are folded in with
// one add-with-carry chain per row: 64 wide products and 64 carry adds.
// (On sm_103a a wide multiply-add costs as much as a high-half multiply, and
// twice a low-half multiply, so separate lo/hi products would cost 1.5x.)
// Squaring: 28 cross products, doubled, plus 8 diagonal squares.  Products
// and reductions live in out-of-line functions (fmul, fsqr): inlining them
// into every call site of a point formula overflows the instruction cache.
// Reduction of the 512-bit product uses the
// special form of p (Solinas, FIPS 186-4 D.2): with 2^256 = 2^224 - 2^192 -
// 2^96 + 1 (mod p), the product c = (c15..c0) reduces to
//     T + 2 S1 + 2 S2 + S3 + S4 - D1 - D2 - D3 - D4       (mod p)
// where each term is an 8-word rearrangement of the c_i (spelled out in
// fe_reduce).  A bias of 5p keeps the intermediate non-negative, after which
// two folds of the top word by 2^256 = K (mod p) bring it below 2^256.
// No multiplications are spent on reduction.
#pragma once
#include <stdint.h>

namespace pcmm {

struct fe {
    uint32_t v[8];
};

// K = 2^256 mod p = 2^224 - 2^192 - 2^96 + 1, little-endian words.
#define PCMM_K0 0x00000001u
#define PCMM_K3 0xffffffffu
#define PCMM_K6 0xfffffffeu

__device__ __forceinline__ void fe_zero(fe& r) {
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = 0;
}

__device__ __forceinline__ void fe_one(fe& r) {
    r.v[0] = 1;
#pragma unroll
    for (int i = 1; i < 8; i++) r.v[i] = 0;
}

// r += mask & K (mask is 0 or 0xffffffff); returns the carry out.
__device__ __forceinline__ uint32_t fe_add_K_masked(fe& r, uint32_t mask) {
    uint32_t k0 = mask & PCMM_K0, k3 = mask, k6 = mask & PCMM_K6, c;
    asm("add.cc.u32  %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.cc.u32 %3, %3, %10;\n\t"
        "addc.cc.u32 %4, %4, %10;\n\t"
        "addc.cc.u32 %5, %5, %10;\n\t"
        "addc.cc.u32 %6, %6, %11;\n\t"
        "addc.cc.u32 %7, %7, 0;\n\t"
        "addc.u32    %8, 0, 0;"
        : "+r"(r.v[0]), "+r"(r.v[1]), "+r"(r.v[2]), "+r"(r.v[3]), "+r"(r.v[4]), "+r"(r.v[5]),
          "+r"(r.v[6]), "+r"(r.v[7]), "=r"(c)
        : "r"(k0), "r"(k3), "r"(k6));
    return c;
}

// r -= mask & K; returns the borrow (1 if it wrapped).
__device__ __forceinline__ uint32_t fe_sub_K_masked(fe& r, uint32_t mask) {
    uint32_t k0 = mask & PCMM_K0, k3 = mask, k6 = mask & PCMM_K6, b;
    asm("sub.cc.u32  %0, %0, %9;\n\t"
        "subc.cc.u32 %1, %1, 0;\n\t"
        "subc.cc.u32 %2, %2, 0;\n\t"
        "subc.cc.u32 %3, %3, %10;\n\t"
        "subc.cc.u32 %4, %4, %10;\n\t"
        "subc.cc.u32 %5, %5, %10;\n\t"
        "subc.cc.u32 %6, %6, %11;\n\t"
        "subc.cc.u32 %7, %7, 0;\n\t"
        "subc.u32    %8, 0, 0;"
        : "+r"(r.v[0]), "+r"(r.v[1]), "+r"(r.v[2]), "+r"(r.v[3]), "+r"(r.v[4]), "+r"(r.v[5]),
          "+r"(r.v[6]), "+r"(r.v[7]), "=r"(b)
        : "r"(k0), "r"(k3), "r"(k6));
    return b & 1u;
}

// r = a + b mod p (weak).  a + b < 2^257; a carry out of 2^256 is replaced by
// adding K = 2^256 mod p.  A second carry (only when the first fold lands at
// or above 2^256, probability about 2^-32) takes a branch.
__device__ __forceinline__ void fe_add(fe& r, const fe& a, const fe& b) {
    uint32_t c;
    asm("add.cc.u32  %0, %9, %17;\n\t"
        "addc.cc.u32 %1, %10, %18;\n\t"
        "addc.cc.u32 %2, %11, %19;\n\t"
        "addc.cc.u32 %3, %12, %20;\n\t"
        "addc.cc.u32 %4, %13, %21;\n\t"
        "addc.cc.u32 %5, %14, %22;\n\t"
        "addc.cc.u32 %6, %15, %23;\n\t"
        "addc.cc.u32 %7, %16, %24;\n\t"
        "addc.u32    %8, 0, 0;"
        : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]),
          "=r"(r.v[6]), "=r"(r.v[7]), "=r"(c)
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
          "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]),
          "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
    c = fe_add_K_masked(r, 0u - c);
    if (c) fe_add_K_masked(r, 0xffffffffu);
}

// r = a - b mod p (weak).  A borrow means the register holds a - b + 2^256;
// subtracting K turns that into a - b + p; a second borrow (only if b - a > p,
// which needs a weakly reduced b >= p) subtracts K again on a branch.
__device__ __forceinline__ void fe_sub(fe& r, const fe& a, const fe& b) {
    uint32_t bw;
    asm("sub.cc.u32  %0, %9, %17;\n\t"
        "subc.cc.u32 %1, %10, %18;\n\t"
        "subc.cc.u32 %2, %11, %19;\n\t"
        "subc.cc.u32 %3, %12, %20;\n\t"
        "subc.cc.u32 %4, %13, %21;\n\t"
        "subc.cc.u32 %5, %14, %22;\n\t"
        "subc.cc.u32 %6, %15, %23;\n\t"
        "subc.cc.u32 %7, %16, %24;\n\t"
        "subc.u32    %8, 0, 0;"
        : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]),
          "=r"(r.v[6]), "=r"(r.v[7]), "=r"(bw)
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
          "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[0]), "r"(b.v[1]), "r"(b.v[2]), "r"(b.v[3]),
          "r"(b.v[4]), "r"(b.v[5]), "r"(b.v[6]), "r"(b.v[7]));
    bw = fe_sub_K_masked(r, bw);
    if (bw) fe_sub_K_masked(r, 0xffffffffu);
}

__device__ __forceinline__ void fe_dbl(fe& r, const fe& a) { fe_add(r, a, a); }

// Canonical representative in [0, p): subtract p once if a >= p.
__device__ __forceinline__ void fe_canon(fe& r, const fe& a) {
    fe t;
    uint32_t bw;
    asm("sub.cc.u32  %0, %9, 0xffffffff;\n\t"
        "subc.cc.u32 %1, %10, 0xffffffff;\n\t"
        "subc.cc.u32 %2, %11, 0xffffffff;\n\t"
        "subc.cc.u32 %3, %12, 0;\n\t"
        "subc.cc.u32 %4, %13, 0;\n\t"
        "subc.cc.u32 %5, %14, 0;\n\t"
        "subc.cc.u32 %6, %15, 1;\n\t"
        "subc.cc.u32 %7, %16, 0xffffffff;\n\t"
        "subc.u32    %8, 0, 0;"
        : "=r"(t.v[0]), "=r"(t.v[1]), "=r"(t.v[2]), "=r"(t.v[3]), "=r"(t.v[4]), "=r"(t.v[5]),
          "=r"(t.v[6]), "=r"(t.v[7]), "=r"(bw)
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
          "r"(a.v[6]), "r"(a.v[7]));
    // bw = 0xffffffff when a < p: keep a.
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = (a.v[i] & bw) | (t.v[i] & ~bw);
}

// True when a = 0 (mod p), i.e. a is 0 or p.
__device__ __forceinline__ bool fe_is_zero(const fe& a) {
    uint32_t z = a.v[0] | a.v[1] | a.v[2] | a.v[3] | a.v[4] | a.v[5] | a.v[6] | a.v[7];
    uint32_t q = (a.v[0] ^ 0xffffffffu) | (a.v[1] ^ 0xffffffffu) | (a.v[2] ^ 0xffffffffu) |
                 a.v[3] | a.v[4] | a.v[5] | (a.v[6] ^ 1u) | (a.v[7] ^ 0xffffffffu);
    return (z == 0u) | (q == 0u);
}

// True when a = b (mod p).
__device__ __forceinline__ bool fe_equal(const fe& a, const fe& b) {
    fe d;
    fe_sub(d, a, b);
    return fe_is_zero(d);
}

// Whether a holds exactly the word representation of 1 (a value of 1 + p,
// which weakly reduced arithmetic could produce, is not recognised; callers
// use this only to skip work when it says yes).
__device__ __forceinline__ bool fe_is_one(const fe& a) {
    uint32_t z = (a.v[0] ^ 1u) | a.v[1] | a.v[2] | a.v[3] | a.v[4] | a.v[5] | a.v[6] | a.v[7];
    return z == 0u;
}

// Reduce the 512-bit value c[0..15] modulo p into r (weak).
__device__ __forceinline__ void fe_reduce(fe& r, const uint32_t c[16]) {
    uint32_t a0, a1, a2, a3, a4, a5, a6, a7, a8;
    uint32_t u3, u4, u5, u6, u7, u8;
    // u = S1 + S2 on words 3..8:  S1 = (c11..c15) at words 3..7,
    //                             S2 = (c12..c15) at words 3..6.
    asm("add.cc.u32  %0, %6, %7;\n\t"
        "addc.cc.u32 %1, %7, %8;\n\t"
        "addc.cc.u32 %2, %8, %9;\n\t"
        "addc.cc.u32 %3, %9, %10;\n\t"
        "addc.cc.u32 %4, %10, 0;\n\t"
        "addc.u32    %5, 0, 0;\n\t"
        // u = 2u
        "add.cc.u32  %0, %0, %0;\n\t"
        "addc.cc.u32 %1, %1, %1;\n\t"
        "addc.cc.u32 %2, %2, %2;\n\t"
        "addc.cc.u32 %3, %3, %3;\n\t"
        "addc.cc.u32 %4, %4, %4;\n\t"
        "addc.u32    %5, %5, %5;"
        : "=r"(u3), "=r"(u4), "=r"(u5), "=r"(u6), "=r"(u7), "=r"(u8)
        : "r"(c[11]), "r"(c[12]), "r"(c[13]), "r"(c[14]), "r"(c[15]));
    // a = T + 5p, with 5p = (4, fffffffb, 5, 0, 0, 4, ffffffff, ffffffff, fffffffb)
    //                       word 8 .................................... word 0
    asm("add.cc.u32  %0, %9, 0xfffffffb;\n\t"
        "addc.cc.u32 %1, %10, 0xffffffff;\n\t"
        "addc.cc.u32 %2, %11, 0xffffffff;\n\t"
        "addc.cc.u32 %3, %12, 4;\n\t"
        "addc.cc.u32 %4, %13, 0;\n\t"
        "addc.cc.u32 %5, %14, 0;\n\t"
        "addc.cc.u32 %6, %15, 5;\n\t"
        "addc.cc.u32 %7, %16, 0xfffffffb;\n\t"
        "addc.u32    %8, 4, 0;"
        : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3), "=r"(a4), "=r"(a5), "=r"(a6), "=r"(a7),
          "=r"(a8)
        : "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(c[5]), "r"(c[6]),
          "r"(c[7]));
    // a += 2 (S1 + S2)
    asm("add.cc.u32  %0, %0, %6;\n\t"
        "addc.cc.u32 %1, %1, %7;\n\t"
        "addc.cc.u32 %2, %2, %8;\n\t"
        "addc.cc.u32 %3, %3, %9;\n\t"
        "addc.cc.u32 %4, %4, %10;\n\t"
        "addc.u32    %5, %5, %11;"
        : "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7), "+r"(a8)
        : "r"(u3), "r"(u4), "r"(u5), "r"(u6), "r"(u7), "r"(u8));
    // a += S3 = (c15, c14, 0, 0, 0, c10, c9, c8)
    // a += S4 = (c8, c13, c15, c14, c13, c11, c10, c9)
    asm("add.cc.u32  %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.cc.u32 %2, %2, %11;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.cc.u32 %4, %4, 0;\n\t"
        "addc.cc.u32 %5, %5, 0;\n\t"
        "addc.cc.u32 %6, %6, %15;\n\t"
        "addc.cc.u32 %7, %7, %16;\n\t"
        "addc.u32    %8, %8, 0;\n\t"
        "add.cc.u32  %0, %0, %10;\n\t"
        "addc.cc.u32 %1, %1, %11;\n\t"
        "addc.cc.u32 %2, %2, %12;\n\t"
        "addc.cc.u32 %3, %3, %14;\n\t"
        "addc.cc.u32 %4, %4, %15;\n\t"
        "addc.cc.u32 %5, %5, %16;\n\t"
        "addc.cc.u32 %6, %6, %14;\n\t"
        "addc.cc.u32 %7, %7, %9;\n\t"
        "addc.u32    %8, %8, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7),
          "+r"(a8)
        : "r"(c[8]), "r"(c[9]), "r"(c[10]), "r"(c[11]), "r"(c[12]), "r"(c[13]), "r"(c[14]),
          "r"(c[15]));
    // a -= D1 = (c10, c8, 0, 0, 0, c13, c12, c11)
    // a -= D2 = (c11, c9, 0, 0, c15, c14, c13, c12)
    asm("sub.cc.u32  %0, %0, %12;\n\t"
        "subc.cc.u32 %1, %1, %13;\n\t"
        "subc.cc.u32 %2, %2, %14;\n\t"
        "subc.cc.u32 %3, %3, 0;\n\t"
        "subc.cc.u32 %4, %4, 0;\n\t"
        "subc.cc.u32 %5, %5, 0;\n\t"
        "subc.cc.u32 %6, %6, %9;\n\t"
        "subc.cc.u32 %7, %7, %11;\n\t"
        "subc.u32    %8, %8, 0;\n\t"
        "sub.cc.u32  %0, %0, %13;\n\t"
        "subc.cc.u32 %1, %1, %14;\n\t"
        "subc.cc.u32 %2, %2, %15;\n\t"
        "subc.cc.u32 %3, %3, %16;\n\t"
        "subc.cc.u32 %4, %4, 0;\n\t"
        "subc.cc.u32 %5, %5, 0;\n\t"
        "subc.cc.u32 %6, %6, %10;\n\t"
        "subc.cc.u32 %7, %7, %12;\n\t"
        "subc.u32    %8, %8, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7),
          "+r"(a8)
        : "r"(c[8]), "r"(c[9]), "r"(c[10]), "r"(c[11]), "r"(c[12]), "r"(c[13]), "r"(c[14]),
          "r"(c[15]));
    // a -= D3 = (c12, 0, c10, c9, c8, c15, c14, c13)
    // a -= D4 = (c13, 0, c11, c10, c9, 0, c15, c14)
    asm("sub.cc.u32  %0, %0, %14;\n\t"
        "subc.cc.u32 %1, %1, %15;\n\t"
        "subc.cc.u32 %2, %2, %16;\n\t"
        "subc.cc.u32 %3, %3, %9;\n\t"
        "subc.cc.u32 %4, %4, %10;\n\t"
        "subc.cc.u32 %5, %5, %11;\n\t"
        "subc.cc.u32 %6, %6, 0;\n\t"
        "subc.cc.u32 %7, %7, %13;\n\t"
        "subc.u32    %8, %8, 0;\n\t"
        "sub.cc.u32  %0, %0, %15;\n\t"
        "subc.cc.u32 %1, %1, %16;\n\t"
        "subc.cc.u32 %2, %2, 0;\n\t"
        "subc.cc.u32 %3, %3, %10;\n\t"
        "subc.cc.u32 %4, %4, %11;\n\t"
        "subc.cc.u32 %5, %5, %12;\n\t"
        "subc.cc.u32 %6, %6, 0;\n\t"
        "subc.cc.u32 %7, %7, %14;\n\t"
        "subc.u32    %8, %8, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7),
          "+r"(a8)
        : "r"(c[8]), "r"(c[9]), "r"(c[10]), "r"(c[11]), "r"(c[12]), "r"(c[13]), "r"(c[14]),
          "r"(c[15]));
    // Now 0 <= a < 12 * 2^256: fold the top word t = a8 with 2^256 = K:
    //   low + t + t 2^224 - t 2^96 - t 2^192.
    uint32_t e1, b1;
    asm("add.cc.u32  %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.cc.u32 %4, %4, 0;\n\t"
        "addc.cc.u32 %5, %5, 0;\n\t"
        "addc.cc.u32 %6, %6, 0;\n\t"
        "addc.cc.u32 %7, %7, %9;\n\t"
        "addc.u32    %8, 0, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7),
          "=r"(e1)
        : "r"(a8));
    asm("sub.cc.u32  %3, %3, %9;\n\t"
        "subc.cc.u32 %4, %4, 0;\n\t"
        "subc.cc.u32 %5, %5, 0;\n\t"
        "subc.cc.u32 %6, %6, %9;\n\t"
        "subc.cc.u32 %7, %7, 0;\n\t"
        "subc.u32    %8, 0, 0;"
        : "+r"(a0), "+r"(a1), "+r"(a2), "+r"(a3), "+r"(a4), "+r"(a5), "+r"(a6), "+r"(a7),
          "=r"(b1)
        : "r"(a8));
    // The folded value is non-negative and below 2^256 + 11 * 2^224, so the
    // net top word e1 + b1 (b1 is 0 or -1) is 0 or 1; it is 1 only when the
    // value reached 2^256 (probability below 2^-27), handled on a branch.
    r.v[0] = a0; r.v[1] = a1; r.v[2] = a2; r.v[3] = a3;
    r.v[4] = a4; r.v[5] = a5; r.v[6] = a6; r.v[7] = a7;
    if (e1 + b1) fe_add_K_masked(r, 0xffffffffu);
}

// t[0..15] = a * b.  Row i: p_j = a_j b_i + t[i+j] (one wide multiply-add,
// never overflowing 64 bits), t[i] = lo(p_0), t[i+j] = lo(p_j) + hi(p_j-1)
// + carry, t[i+8] = hi(p_7) + carry.
__device__ __forceinline__ void mul_wide(uint32_t t[16], const fe& a, const fe& b) {
    uint64_t p[8];
#pragma unroll
    for (int j = 0; j < 8; j++) p[j] = (uint64_t)a.v[j] * b.v[0];
    t[0] = (uint32_t)p[0];
    asm("add.cc.u32 %0, %8, %15;\n\taddc.cc.u32 %1, %9, %16;\n\taddc.cc.u32 %2, %10, %17;\n\t"
        "addc.cc.u32 %3, %11, %18;\n\taddc.cc.u32 %4, %12, %19;\n\taddc.cc.u32 %5, %13, %20;\n\t"
        "addc.cc.u32 %6, %14, %21;\n\taddc.u32 %7, %22, 0;"
        : "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]), "=r"(t[7]), "=r"(t[8])
        : "r"((uint32_t)p[1]), "r"((uint32_t)p[2]), "r"((uint32_t)p[3]), "r"((uint32_t)p[4]), "r"((uint32_t)p[5]),
          "r"((uint32_t)p[6]), "r"((uint32_t)p[7]), "r"((uint32_t)(p[0] >> 32)), "r"((uint32_t)(p[1] >> 32)),
          "r"((uint32_t)(p[2] >> 32)), "r"((uint32_t)(p[3] >> 32)), "r"((uint32_t)(p[4] >> 32)),
          "r"((uint32_t)(p[5] >> 32)), "r"((uint32_t)(p[6] >> 32)), "r"((uint32_t)(p[7] >> 32)));
#pragma unroll
    for (int i = 1; i < 8; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) p[j] = (uint64_t)a.v[j] * b.v[i] + t[i + j];
        t[i] = (uint32_t)p[0];
        asm("add.cc.u32 %0, %8, %15;\n\taddc.cc.u32 %1, %9, %16;\n\taddc.cc.u32 %2, %10, %17;\n\t"
            "addc.cc.u32 %3, %11, %18;\n\taddc.cc.u32 %4, %12, %19;\n\taddc.cc.u32 %5, %13, %20;\n\t"
            "addc.cc.u32 %6, %14, %21;\n\taddc.u32 %7, %22, 0;"
            : "=r"(t[i + 1]), "=r"(t[i + 2]), "=r"(t[i + 3]), "=r"(t[i + 4]), "=r"(t[i + 5]), "=r"(t[i + 6]),
              "=r"(t[i + 7]), "=r"(t[i + 8])
            : "r"((uint32_t)p[1]), "r"((uint32_t)p[2]), "r"((uint32_t)p[3]), "r"((uint32_t)p[4]), "r"((uint32_t)p[5]),
              "r"((uint32_t)p[6]), "r"((uint32_t)p[7]), "r"((uint32_t)(p[0] >> 32)), "r"((uint32_t)(p[1] >> 32)),
              "r"((uint32_t)(p[2] >> 32)), "r"((uint32_t)(p[3] >> 32)), "r"((uint32_t)(p[4] >> 32)),
              "r"((uint32_t)(p[5] >> 32)), "r"((uint32_t)(p[6] >> 32)), "r"((uint32_t)(p[7] >> 32)));
    }
}

// out[k] = lo[k] + hi[k] + carry (k < N), out[N] = hi[N] + carry: one carry
// chain, kept inside a single asm statement so the carry flag survives.
template <int N> __device__ __forceinline__ void chain_add(uint32_t* out, const uint32_t* lo, const uint32_t* hi);
template <> __device__ __forceinline__ void chain_add<1>(uint32_t* out, const uint32_t* lo, const uint32_t* hi) {
    asm("add.cc.u32  %0, %2, %3;\n\t"
        "addc.u32 %1, %4, 0;"
        : "=r"(out[0]), "=r"(out[1])
        : "r"(lo[0]), "r"(hi[0]), "r"(hi[1]));
}
template <> __device__ __forceinline__ void chain_add<2>(uint32_t* out, const uint32_t* lo, const uint32_t* hi) {
    asm("add.cc.u32  %0, %3, %5;\n\t"
        "addc.cc.u32 %1, %4, %6;\n\t"
        "addc.u32 %2, %7, 0;"
        : "=r"(out[0]), "=r"(out[1]), "=r"(out[2])
        : "r"(lo[0]), "r"(lo[1]), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]));
}
template <> __device__ __forceinline__ void chain_add<3>(uint32_t* out, const uint32_t* lo, const uint32_t* hi) {
    asm("add.cc.u32  %0, %4, %7;\n\t"
        "addc.cc.u32 %1, %5, %8;\n\t"
        "addc.cc.u32 %2, %6, %9;\n\t"
        "addc.u32 %3, %10, 0;"
        : "=r"(out[0]), "=r"(out[1]), "=r"(out[2]), "=r"(out[3])
        : "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]));
}
template <> __device__ __forceinline__ void chain_add<4>(uint32_t* out, const uint32_t* lo, const uint32_t* hi) {
    asm("add.cc.u32  %0, %5, %9;\n\t"
        "addc.cc.u32 %1, %6, %10;\n\t"
        "addc.cc.u32 %2, %7, %11;\n\t"
        "addc.cc.u32 %3, %8, %12;\n\t"
        "addc.u32 %4, %13, 0;"
        : "=r"(out[0]), "=r"(out[1]), "=r"(out[2]), "=r"(out[3]), "=r"(out[4])
        : "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]));
}
template <> __device__ __forceinline__ void chain_add<5>(uint32_t* out, const uint32_t* lo, const uint32_t* hi) {
    asm("add.cc.u32  %0, %6, %11;\n\t"
        "addc.cc.u32 %1, %7, %12;\n\t"
        "addc.cc.u32 %2, %8, %13;\n\t"
        "addc.cc.u32 %3, %9, %14;\n\t"
        "addc.cc.u32 %4, %10, %15;\n\t"
        "addc.u32 %5, %16, 0;"
        : "=r"(out[0]), "=r"(out[1]), "=r"(out[2]), "=r"(out[3]), "=r"(out[4]), "=r"(out[5])
        : "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]));
}
template <> __device__ __forceinline__ void chain_add<6>(uint32_t* out, const uint32_t* lo, const uint32_t* hi) {
    asm("add.cc.u32  %0, %7, %13;\n\t"
        "addc.cc.u32 %1, %8, %14;\n\t"
        "addc.cc.u32 %2, %9, %15;\n\t"
        "addc.cc.u32 %3, %10, %16;\n\t"
        "addc.cc.u32 %4, %11, %17;\n\t"
        "addc.cc.u32 %5, %12, %18;\n\t"
        "addc.u32 %6, %19, 0;"
        : "=r"(out[0]), "=r"(out[1]), "=r"(out[2]), "=r"(out[3]), "=r"(out[4]), "=r"(out[5]), "=r"(out[6])
        : "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]));
}
template <> __device__ __forceinline__ void chain_add<7>(uint32_t* out, const uint32_t* lo, const uint32_t* hi) {
    asm("add.cc.u32  %0, %8, %15;\n\t"
        "addc.cc.u32 %1, %9, %16;\n\t"
        "addc.cc.u32 %2, %10, %17;\n\t"
        "addc.cc.u32 %3, %11, %18;\n\t"
        "addc.cc.u32 %4, %12, %19;\n\t"
        "addc.cc.u32 %5, %13, %20;\n\t"
        "addc.cc.u32 %6, %14, %21;\n\t"
        "addc.u32 %7, %22, 0;"
        : "=r"(out[0]), "=r"(out[1]), "=r"(out[2]), "=r"(out[3]), "=r"(out[4]), "=r"(out[5]), "=r"(out[6]), "=r"(out[7])
        : "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3]), "r"(lo[4]), "r"(lo[5]), "r"(lo[6]), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]), "r"(hi[3]), "r"(hi[4]), "r"(hi[5]), "r"(hi[6]), "r"(hi[7]));
}

// Squaring with wide products: cross products row by row, doubled, plus squares.
__device__ __forceinline__ void sqr_wide(uint32_t t[16], const fe& a) {
    uint32_t lo[8], hi[8];
    // row 0: a0 * a1..a7 -> t[1..8]
#pragma unroll
    for (int j = 1; j < 8; j++) {
        uint64_t p = (uint64_t)a.v[0] * a.v[j];
        lo[j] = (uint32_t)p; hi[j] = (uint32_t)(p >> 32);
    }
    t[1] = lo[1];
    chain_add<6>(&t[2], &lo[2], &hi[1]);
#define SQROW(I)                                                        \
    {                                                                   \
        _Pragma("unroll") for (int j = I + 1; j < 8; j++) {             \
            uint64_t p = (uint64_t)a.v[I] * a.v[j] + t[I + j];          \
            lo[j] = (uint32_t)p; hi[j] = (uint32_t)(p >> 32);           \
        }                                                               \
        t[2 * I + 1] = lo[I + 1];                                       \
        chain_add<6 - I>(&t[2 * I + 2], &lo[I + 2], &hi[I + 1]);        \
    }
    SQROW(1) SQROW(2) SQROW(3) SQROW(4) SQROW(5)
#undef SQROW
    {
        uint64_t p = (uint64_t)a.v[6] * a.v[7] + t[13];
        t[13] = (uint32_t)p;
        t[14] = (uint32_t)(p >> 32);
    }
    // double u[1..14] and add the squares a_i^2 at 2i
    uint64_t d[8];
#pragma unroll
    for (int i = 0; i < 8; i++) d[i] = (uint64_t)a.v[i] * a.v[i];
    asm("add.cc.u32  %1, %1, %1;\n\t"
        "addc.cc.u32 %2, %2, %2;\n\t"
        "addc.cc.u32 %3, %3, %3;\n\t"
        "addc.cc.u32 %4, %4, %4;\n\t"
        "addc.cc.u32 %5, %5, %5;\n\t"
        "addc.cc.u32 %6, %6, %6;\n\t"
        "addc.cc.u32 %7, %7, %7;\n\t"
        "addc.cc.u32 %8, %8, %8;\n\t"
        "addc.cc.u32 %9, %9, %9;\n\t"
        "addc.cc.u32 %10, %10, %10;\n\t"
        "addc.cc.u32 %11, %11, %11;\n\t"
        "addc.cc.u32 %12, %12, %12;\n\t"
        "addc.cc.u32 %13, %13, %13;\n\t"
        "addc.cc.u32 %14, %14, %14;\n\t"
        "addc.u32    %15, 0, 0;\n\t"
        "mov.b32     %0, %16;\n\t"
        "add.cc.u32  %1, %1, %17;\n\t"
        "addc.cc.u32 %2, %2, %18;\n\t"
        "addc.cc.u32 %3, %3, %19;\n\t"
        "addc.cc.u32 %4, %4, %20;\n\t"
        "addc.cc.u32 %5, %5, %21;\n\t"
        "addc.cc.u32 %6, %6, %22;\n\t"
        "addc.cc.u32 %7, %7, %23;\n\t"
        "addc.cc.u32 %8, %8, %24;\n\t"
        "addc.cc.u32 %9, %9, %25;\n\t"
        "addc.cc.u32 %10, %10, %26;\n\t"
        "addc.cc.u32 %11, %11, %27;\n\t"
        "addc.cc.u32 %12, %12, %28;\n\t"
        "addc.cc.u32 %13, %13, %29;\n\t"
        "addc.cc.u32 %14, %14, %30;\n\t"
        "addc.u32    %15, %15, %31;"
        : "=r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]),
          "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]), "+r"(t[13]), "+r"(t[14]), "=r"(t[15])
        : "r"((uint32_t)d[0]), "r"((uint32_t)(d[0] >> 32)), "r"((uint32_t)d[1]), "r"((uint32_t)(d[1] >> 32)),
          "r"((uint32_t)d[2]), "r"((uint32_t)(d[2] >> 32)), "r"((uint32_t)d[3]), "r"((uint32_t)(d[3] >> 32)),
          "r"((uint32_t)d[4]), "r"((uint32_t)(d[4] >> 32)), "r"((uint32_t)d[5]), "r"((uint32_t)(d[5] >> 32)),
          "r"((uint32_t)d[6]), "r"((uint32_t)(d[6] >> 32)), "r"((uint32_t)d[7]), "r"((uint32_t)(d[7] >> 32)));
}

__device__ __forceinline__ void fe_mul(fe& r, const fe& a, const fe& b) {
    uint32_t t[16];
    mul_wide(t, a, b);
    fe_reduce(r, t);
}

__device__ __forceinline__ void fe_sqr(fe& r, const fe& a) {
    uint32_t t[16];
    sqr_wide(t, a);
    fe_reduce(r, t);
}

// Out-of-line multiplication and squaring (by value): the hot point formulas
// call these so that one copy of the product and reduction code serves every
// call site.
static __device__ __noinline__ fe fmul(fe a, fe b) {
    fe r;
    fe_mul(r, a, b);
    return r;
}

static __device__ __noinline__ fe fsqr(fe a) {
    fe r;
    fe_sqr(r, a);
    return r;
}

// x <- x 2^-k mod p for canonical x and 1 <= k <= 31.  Since p = -1 mod
// 2^32, x + (x mod 2^k) p is a multiple of 2^k, below 2^k p, so the shifted
// sum is canonical again.
__device__ __forceinline__ void fe_div_pow2(fe& x, unsigned k) {
    const uint32_t q = x.v[0] & ((1u << k) - 1u);
    // t = x + q p with p = 2^256 - 2^224 + 2^192 + 2^96 - 1 (words 0..7:
    // ffffffff x3, 0 x2, 1, ffffffff; the 2^256 term lands in word 8).
    uint32_t t[9];
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint64_t pj = (j < 3 || j == 7) ? 0xffffffffull : (j == 6 ? 1ull : 0ull);
        c += (uint64_t)x.v[j] + (uint64_t)q * pj;
        t[j] = (uint32_t)c;
        c >>= 32;
    }
    t[8] = (uint32_t)c;
#pragma unroll
    for (int j = 0; j < 8; j++) x.v[j] = __funnelshift_r(t[j], t[j + 1], k);
}

// r = a^-1 mod p for a != 0 mod p (0 gives 0), a weakly reduced; r is
// canonical.  Binary extended Euclid: with u = a, v = p, x1 = 1, x2 = 0 the
// invariants x1 a = u and x2 a = v (mod p) hold throughout; factors of two
// leave u (or v) together with the same power of two from x1 (or x2), and
// the smaller of two odd u, v is subtracted from the larger (their
// difference is even), until one of them is 1.  About 2 log2 p steps of a
// few 256-bit additions each, against the 267 dependent multiplications of
// a Fermat power.
static __device__ __noinline__ void fe_inv(fe& r, const fe& a) {
    fe u, v, x1, x2;
    fe_canon(u, a);
    if ((u.v[0] | u.v[1] | u.v[2] | u.v[3] | u.v[4] | u.v[5] | u.v[6] | u.v[7]) == 0u) {
        fe_zero(r);
        return;
    }
    v.v[0] = v.v[1] = v.v[2] = 0xffffffffu;
    v.v[3] = v.v[4] = v.v[5] = 0u;
    v.v[6] = 1u;
    v.v[7] = 0xffffffffu;
    fe_one(x1);
    fe_zero(x2);
    // Each step removes a factor of two or shrinks u + v: the bound is never
    // reached for a != 0 mod p.
    for (int it = 0; it < 4096; it++) {
        const bool u1 = ((u.v[0] ^ 1u) | u.v[1] | u.v[2] | u.v[3] | u.v[4] | u.v[5] | u.v[6] | u.v[7]) == 0u;
        if (u1) break;
        const bool v1 = ((v.v[0] ^ 1u) | v.v[1] | v.v[2] | v.v[3] | v.v[4] | v.v[5] | v.v[6] | v.v[7]) == 0u;
        if (v1) {
            x1 = x2;
            break;
        }
        if (!(u.v[0] & 1u)) {
            const unsigned k = u.v[0] ? (unsigned)(__ffs(u.v[0]) - 1) : 31u;
#pragma unroll
            for (int j = 0; j < 7; j++) u.v[j] = __funnelshift_r(u.v[j], u.v[j + 1], k);
            u.v[7] >>= k;
            fe_div_pow2(x1, k);
            continue;
        }
        if (!(v.v[0] & 1u)) {
            const unsigned k = v.v[0] ? (unsigned)(__ffs(v.v[0]) - 1) : 31u;
#pragma unroll
            for (int j = 0; j < 7; j++) v.v[j] = __funnelshift_r(v.v[j], v.v[j + 1], k);
            v.v[7] >>= k;
            fe_div_pow2(x2, k);
            continue;
        }
        // d = u - v; if no borrow u <- d, x1 <- x1 - x2, else v <- -d, x2 <- x2 - x1.
        fe d;
        uint32_t bw;
        asm("sub.cc.u32  %0, %9, %17;\n\t"
            "subc.cc.u32 %1, %10, %18;\n\t"
            "subc.cc.u32 %2, %11, %19;\n\t"
            "subc.cc.u32 %3, %12, %20;\n\t"
            "subc.cc.u32 %4, %13, %21;\n\t"
            "subc.cc.u32 %5, %14, %22;\n\t"
            "subc.cc.u32 %6, %15, %23;\n\t"
            "subc.cc.u32 %7, %16, %24;\n\t"
            "subc.u32    %8, 0, 0;"
            : "=r"(d.v[0]), "=r"(d.v[1]), "=r"(d.v[2]), "=r"(d.v[3]), "=r"(d.v[4]), "=r"(d.v[5]),
              "=r"(d.v[6]), "=r"(d.v[7]), "=r"(bw)
            : "r"(u.v[0]), "r"(u.v[1]), "r"(u.v[2]), "r"(u.v[3]), "r"(u.v[4]), "r"(u.v[5]), "r"(u.v[6]),
              "r"(u.v[7]), "r"(v.v[0]), "r"(v.v[1]), "r"(v.v[2]), "r"(v.v[3]), "r"(v.v[4]), "r"(v.v[5]),
              "r"(v.v[6]), "r"(v.v[7]));
        if (!bw) {
            u = d;
            fe_sub(x1, x1, x2);
            fe_canon(x1, x1);
        } else {
            asm("sub.cc.u32  %0, 0, %0;\n\t"
                "subc.cc.u32 %1, 0, %1;\n\t"
                "subc.cc.u32 %2, 0, %2;\n\t"
                "subc.cc.u32 %3, 0, %3;\n\t"
                "subc.cc.u32 %4, 0, %4;\n\t"
                "subc.cc.u32 %5, 0, %5;\n\t"
                "subc.cc.u32 %6, 0, %6;\n\t"
                "subc.u32    %7, 0, %7;"
                : "+r"(d.v[0]), "+r"(d.v[1]), "+r"(d.v[2]), "+r"(d.v[3]), "+r"(d.v[4]), "+r"(d.v[5]),
                  "+r"(d.v[6]), "+r"(d.v[7]));
            v = d;
            fe_sub(x2, x2, x1);
            fe_canon(x2, x2);
        }
    }
    r = x1;
}

// r = a b - c d (mod p) with a single reduction: the two 512-bit products
// are subtracted, p 2^256 (= 0 mod p) is added back while the difference is
// negative (once, or on a rare branch twice), then the sum is reduced.
__device__ __forceinline__ fe fe_mulsub(const fe& a, const fe& b, const fe& c, const fe& d) {
    uint32_t u[16], v[16];
    mul_wide(u, a, b);
    mul_wide(v, c, d);
    uint32_t bw;
    asm("sub.cc.u32  %0, %0, %17;\n\t"
        "subc.cc.u32 %1, %1, %18;\n\t"
        "subc.cc.u32 %2, %2, %19;\n\t"
        "subc.cc.u32 %3, %3, %20;\n\t"
        "subc.cc.u32 %4, %4, %21;\n\t"
        "subc.cc.u32 %5, %5, %22;\n\t"
        "subc.cc.u32 %6, %6, %23;\n\t"
        "subc.cc.u32 %7, %7, %24;\n\t"
        "subc.cc.u32 %8, %8, %25;\n\t"
        "subc.cc.u32 %9, %9, %26;\n\t"
        "subc.cc.u32 %10, %10, %27;\n\t"
        "subc.cc.u32 %11, %11, %28;\n\t"
        "subc.cc.u32 %12, %12, %29;\n\t"
        "subc.cc.u32 %13, %13, %30;\n\t"
        "subc.cc.u32 %14, %14, %31;\n\t"
        "subc.cc.u32 %15, %15, %32;\n\t"
        "subc.u32    %16, 0, 0;"
        : "+r"(u[0]), "+r"(u[1]), "+r"(u[2]), "+r"(u[3]), "+r"(u[4]), "+r"(u[5]), "+r"(u[6]), "+r"(u[7]),
          "+r"(u[8]), "+r"(u[9]), "+r"(u[10]), "+r"(u[11]), "+r"(u[12]), "+r"(u[13]), "+r"(u[14]),
          "+r"(u[15]), "=r"(bw)
        : "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
          "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]));
    // On a borrow (bw = 0xffffffff) add p to the high half.
    uint32_t c2;
    asm("add.cc.u32  %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.cc.u32 %2, %2, %9;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.cc.u32 %4, %4, 0;\n\t"
        "addc.cc.u32 %5, %5, 0;\n\t"
        "addc.cc.u32 %6, %6, %10;\n\t"
        "addc.cc.u32 %7, %7, %9;\n\t"
        "addc.u32    %8, 0, 0;"
        : "+r"(u[8]), "+r"(u[9]), "+r"(u[10]), "+r"(u[11]), "+r"(u[12]), "+r"(u[13]), "+r"(u[14]),
          "+r"(u[15]), "=r"(c2)
        : "r"(bw), "r"(bw & 1u));
    if (bw && !c2) {  // still negative (needs c d - a b > p 2^256): add p 2^256 again
        asm("add.cc.u32  %0, %0, 0xffffffff;\n\t"
            "addc.cc.u32 %1, %1, 0xffffffff;\n\t"
            "addc.cc.u32 %2, %2, 0xffffffff;\n\t"
            "addc.cc.u32 %3, %3, 0;\n\t"
            "addc.cc.u32 %4, %4, 0;\n\t"
            "addc.cc.u32 %5, %5, 0;\n\t"
            "addc.cc.u32 %6, %6, 1;\n\t"
            "addc.u32    %7, %7, 0xffffffff;"
            : "+r"(u[8]), "+r"(u[9]), "+r"(u[10]), "+r"(u[11]), "+r"(u[12]), "+r"(u[13]), "+r"(u[14]),
              "+r"(u[15]));
    }
    fe r;
    fe_reduce(r, u);
    return r;
}

static __device__ __noinline__ fe fmulsub(fe a, fe b, fe c, fe d) { return fe_mulsub(a, b, c, d); }

// Multiplication, squaring and a b - c d either out of line (INL = false:
// one shared copy of the code) or inlined at the call site (INL = true).
template <bool INL>
__device__ __forceinline__ fe mul_t(const fe& a, const fe& b) {
    if (INL) {
        fe r;
        fe_mul(r, a, b);
        return r;
    }
    return fmul(a, b);
}
template <bool INL>
__device__ __forceinline__ fe sqr_t(const fe& a) {
    if (INL) {
        fe r;
        fe_sqr(r, a);
        return r;
    }
    return fsqr(a);
}
template <bool INL>
__device__ __forceinline__ fe mulsub_t(const fe& a, const fe& b, const fe& c, const fe& d) {
    if (INL) return fe_mulsub(a, b, c, d);
    return fmulsub(a, b, c, d);
}

}  // namespace pcmm
