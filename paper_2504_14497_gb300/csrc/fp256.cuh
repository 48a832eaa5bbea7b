// Prime-field arithmetic in F_p for NIST P-256, p = 2^256 - 2^224 + 2^192 + 2^96 - 1
// (Section 4.1), on sm_103a.
//
// Representation: 8 x 32-bit little-endian limbs held in registers.  Values
// are kept WEAKLY reduced: any integer in [0, 2^256) that is congruent to the
// field element (so 0 may appear as 0 or as p).  fe_canon() gives the unique
// representative below p; it is applied only when a result leaves the
// library or when a value must be compared.
//
// Multiplication: 8x8-limb operand scanning with mad.lo/madc.hi carry chains
// (64 limb products = 128 IMAD); squaring: 28 cross products doubled plus 8
// diagonal squares (72 IMAD).  Reduction of the 512-bit product uses the
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

// r = a + b mod p (weak).  a + b < 2^257; each carry out of 2^256 is
// replaced by adding K; at most two folds are needed.
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
    fe_add_K_masked(r, 0u - c);
}

// r = a - b mod p (weak).  A borrow means the register holds a - b + 2^256;
// subtracting K turns that into a - b + p; a second borrow (b - a > p)
// subtracts K again, giving a - b + 2p.
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
    bw = fe_sub_K_masked(r, bw);  // bw is 0 or 0xffffffff
    fe_sub_K_masked(r, 0u - bw);
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
    // net top word e1 + b1 (b1 is 0 or -1) is 0 or 1; one more fold suffices.
    r.v[0] = a0; r.v[1] = a1; r.v[2] = a2; r.v[3] = a3;
    r.v[4] = a4; r.v[5] = a5; r.v[6] = a6; r.v[7] = a7;
    fe_add_K_masked(r, 0u - (e1 + b1));
}

// t[0..15] = a * b, operand scanning, one carry chain pair per row.
__device__ __forceinline__ void mul_wide(uint32_t t[16], const fe& a, const fe& b) {
    // Row 0.
    asm("mul.lo.u32     %0, %9, %17;\n\t"
        "mul.lo.u32     %1, %10, %17;\n\t"
        "mul.lo.u32     %2, %11, %17;\n\t"
        "mul.lo.u32     %3, %12, %17;\n\t"
        "mul.lo.u32     %4, %13, %17;\n\t"
        "mul.lo.u32     %5, %14, %17;\n\t"
        "mul.lo.u32     %6, %15, %17;\n\t"
        "mul.lo.u32     %7, %16, %17;\n\t"
        "mad.hi.cc.u32  %1, %9, %17, %1;\n\t"
        "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
        "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
        "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
        "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
        "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
        "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
        "madc.hi.u32    %8, %16, %17, 0;"
        : "=r"(t[0]), "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]),
          "=r"(t[7]), "=r"(t[8])
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
          "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[0]));
    // Rows 1..7: t[i..i+7] += lo(a b_i), carry into the new word t[i+8],
    // then t[i+1..i+8] += hi(a b_i).  The partial sum is below 2^(32(i+9)),
    // so the final hi chain cannot carry out.
#pragma unroll
    for (int i = 1; i < 8; i++) {
        asm("mad.lo.cc.u32  %0, %9, %17, %0;\n\t"
            "madc.lo.cc.u32 %1, %10, %17, %1;\n\t"
            "madc.lo.cc.u32 %2, %11, %17, %2;\n\t"
            "madc.lo.cc.u32 %3, %12, %17, %3;\n\t"
            "madc.lo.cc.u32 %4, %13, %17, %4;\n\t"
            "madc.lo.cc.u32 %5, %14, %17, %5;\n\t"
            "madc.lo.cc.u32 %6, %15, %17, %6;\n\t"
            "madc.lo.cc.u32 %7, %16, %17, %7;\n\t"
            "addc.u32       %8, 0, 0;\n\t"
            "mad.hi.cc.u32  %1, %9, %17, %1;\n\t"
            "madc.hi.cc.u32 %2, %10, %17, %2;\n\t"
            "madc.hi.cc.u32 %3, %11, %17, %3;\n\t"
            "madc.hi.cc.u32 %4, %12, %17, %4;\n\t"
            "madc.hi.cc.u32 %5, %13, %17, %5;\n\t"
            "madc.hi.cc.u32 %6, %14, %17, %6;\n\t"
            "madc.hi.cc.u32 %7, %15, %17, %7;\n\t"
            "madc.hi.u32    %8, %16, %17, %8;"
            : "+r"(t[i]), "+r"(t[i + 1]), "+r"(t[i + 2]), "+r"(t[i + 3]), "+r"(t[i + 4]),
              "+r"(t[i + 5]), "+r"(t[i + 6]), "+r"(t[i + 7]), "=r"(t[i + 8])
            : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
              "r"(a.v[6]), "r"(a.v[7]), "r"(b.v[i]));
    }
}

// t[0..15] = a^2: cross products a_i a_j (i < j) doubled, plus the squares.
__device__ __forceinline__ void sqr_wide(uint32_t t[16], const fe& a) {
    // Cross products into t[1..14]; t[0] = t[15] = 0 for now.
    // Row 0: a0 * a1..a7 at words 1..8.
    asm("mul.lo.u32     %0, %8, %9;\n\t"
        "mul.lo.u32     %1, %8, %10;\n\t"
        "mul.lo.u32     %2, %8, %11;\n\t"
        "mul.lo.u32     %3, %8, %12;\n\t"
        "mul.lo.u32     %4, %8, %13;\n\t"
        "mul.lo.u32     %5, %8, %14;\n\t"
        "mul.lo.u32     %6, %8, %15;\n\t"
        "mad.hi.cc.u32  %1, %8, %9, %1;\n\t"
        "madc.hi.cc.u32 %2, %8, %10, %2;\n\t"
        "madc.hi.cc.u32 %3, %8, %11, %3;\n\t"
        "madc.hi.cc.u32 %4, %8, %12, %4;\n\t"
        "madc.hi.cc.u32 %5, %8, %13, %5;\n\t"
        "madc.hi.cc.u32 %6, %8, %14, %6;\n\t"
        "madc.hi.u32    %7, %8, %15, 0;"
        : "=r"(t[1]), "=r"(t[2]), "=r"(t[3]), "=r"(t[4]), "=r"(t[5]), "=r"(t[6]), "=r"(t[7]),
          "=r"(t[8])
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
          "r"(a.v[6]), "r"(a.v[7]));
    // Row 1: a1 * a2..a7 at words 3..9.
    asm("mad.lo.cc.u32  %0, %7, %8, %0;\n\t"
        "madc.lo.cc.u32 %1, %7, %9, %1;\n\t"
        "madc.lo.cc.u32 %2, %7, %10, %2;\n\t"
        "madc.lo.cc.u32 %3, %7, %11, %3;\n\t"
        "madc.lo.cc.u32 %4, %7, %12, %4;\n\t"
        "madc.lo.cc.u32 %5, %7, %13, %5;\n\t"
        "addc.u32       %6, 0, 0;\n\t"
        "mad.hi.cc.u32  %1, %7, %8, %1;\n\t"
        "madc.hi.cc.u32 %2, %7, %9, %2;\n\t"
        "madc.hi.cc.u32 %3, %7, %10, %3;\n\t"
        "madc.hi.cc.u32 %4, %7, %11, %4;\n\t"
        "madc.hi.cc.u32 %5, %7, %12, %5;\n\t"
        "madc.hi.u32    %6, %7, %13, %6;"
        : "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "=r"(t[9])
        : "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]),
          "r"(a.v[7]));
    // Row 2: a2 * a3..a7 at words 5..10.
    asm("mad.lo.cc.u32  %0, %6, %7, %0;\n\t"
        "madc.lo.cc.u32 %1, %6, %8, %1;\n\t"
        "madc.lo.cc.u32 %2, %6, %9, %2;\n\t"
        "madc.lo.cc.u32 %3, %6, %10, %3;\n\t"
        "madc.lo.cc.u32 %4, %6, %11, %4;\n\t"
        "addc.u32       %5, 0, 0;\n\t"
        "mad.hi.cc.u32  %1, %6, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %6, %8, %2;\n\t"
        "madc.hi.cc.u32 %3, %6, %9, %3;\n\t"
        "madc.hi.cc.u32 %4, %6, %10, %4;\n\t"
        "madc.hi.u32    %5, %6, %11, %5;"
        : "+r"(t[5]), "+r"(t[6]), "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "=r"(t[10])
        : "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
    // Row 3: a3 * a4..a7 at words 7..11.
    asm("mad.lo.cc.u32  %0, %5, %6, %0;\n\t"
        "madc.lo.cc.u32 %1, %5, %7, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %8, %2;\n\t"
        "madc.lo.cc.u32 %3, %5, %9, %3;\n\t"
        "addc.u32       %4, 0, 0;\n\t"
        "mad.hi.cc.u32  %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.cc.u32 %3, %5, %8, %3;\n\t"
        "madc.hi.u32    %4, %5, %9, %4;"
        : "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "=r"(t[11])
        : "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
    // Row 4: a4 * a5..a7 at words 9..12.
    asm("mad.lo.cc.u32  %0, %4, %5, %0;\n\t"
        "madc.lo.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32       %3, 0, 0;\n\t"
        "mad.hi.cc.u32  %1, %4, %5, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %6, %2;\n\t"
        "madc.hi.u32    %3, %4, %7, %3;"
        : "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "=r"(t[12])
        : "r"(a.v[4]), "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
    // Row 5: a5 * a6..a7 at words 11..13.
    asm("mad.lo.cc.u32  %0, %3, %4, %0;\n\t"
        "madc.lo.cc.u32 %1, %3, %5, %1;\n\t"
        "addc.u32       %2, 0, 0;\n\t"
        "mad.hi.cc.u32  %1, %3, %4, %1;\n\t"
        "madc.hi.u32    %2, %3, %5, %2;"
        : "+r"(t[11]), "+r"(t[12]), "=r"(t[13])
        : "r"(a.v[5]), "r"(a.v[6]), "r"(a.v[7]));
    // Row 6: a6 * a7 at words 13..14.
    asm("mad.lo.cc.u32  %0, %2, %3, %0;\n\t"
        "madc.hi.u32    %1, %2, %3, 0;"
        : "+r"(t[13]), "=r"(t[14])
        : "r"(a.v[6]), "r"(a.v[7]));
    // Double the cross products and add the diagonal squares a_i^2 at 2i.
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
        "mul.lo.u32     %0, %16, %16;\n\t"
        "mad.hi.cc.u32  %1, %16, %16, %1;\n\t"
        "madc.lo.cc.u32 %2, %17, %17, %2;\n\t"
        "madc.hi.cc.u32 %3, %17, %17, %3;\n\t"
        "madc.lo.cc.u32 %4, %18, %18, %4;\n\t"
        "madc.hi.cc.u32 %5, %18, %18, %5;\n\t"
        "madc.lo.cc.u32 %6, %19, %19, %6;\n\t"
        "madc.hi.cc.u32 %7, %19, %19, %7;\n\t"
        "madc.lo.cc.u32 %8, %20, %20, %8;\n\t"
        "madc.hi.cc.u32 %9, %20, %20, %9;\n\t"
        "madc.lo.cc.u32 %10, %21, %21, %10;\n\t"
        "madc.hi.cc.u32 %11, %21, %21, %11;\n\t"
        "madc.lo.cc.u32 %12, %22, %22, %12;\n\t"
        "madc.hi.cc.u32 %13, %22, %22, %13;\n\t"
        "madc.lo.cc.u32 %14, %23, %23, %14;\n\t"
        "madc.hi.u32    %15, %23, %23, %15;"
        : "=r"(t[0]), "+r"(t[1]), "+r"(t[2]), "+r"(t[3]), "+r"(t[4]), "+r"(t[5]), "+r"(t[6]),
          "+r"(t[7]), "+r"(t[8]), "+r"(t[9]), "+r"(t[10]), "+r"(t[11]), "+r"(t[12]),
          "+r"(t[13]), "+r"(t[14]), "=r"(t[15])
        : "r"(a.v[0]), "r"(a.v[1]), "r"(a.v[2]), "r"(a.v[3]), "r"(a.v[4]), "r"(a.v[5]),
          "r"(a.v[6]), "r"(a.v[7]));
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

__device__ __forceinline__ void fe_sqr_n(fe& r, const fe& a, int n) {
    fe_sqr(r, a);
    for (int i = 1; i < n; i++) fe_sqr(r, r);
}

// r = a^(p-2) = a^-1 for a != 0 (Fermat).  Addition chain over the runs of
// ones in p - 2 = ffffffff 00000001 00000000^3 ffffffff ffffffff fffffffd
// (hex, high to low): with x_k = a^(2^k - 1), build x2, x3, x6, x12, x15,
// x30, x32, then 255 squarings and 12 multiplications in total.
static __device__ __noinline__ void fe_inv(fe& r, const fe& a) {
    fe x2, x3, x6, x12, x15, x30, x32, t;
    fe_sqr(t, a);       fe_mul(x2, t, a);      // 2^2 - 1
    fe_sqr(t, x2);      fe_mul(x3, t, a);      // 2^3 - 1
    fe_sqr_n(t, x3, 3); fe_mul(x6, t, x3);     // 2^6 - 1
    fe_sqr_n(t, x6, 6); fe_mul(x12, t, x6);    // 2^12 - 1
    fe_sqr_n(t, x12, 3); fe_mul(x15, t, x3);   // 2^15 - 1
    fe_sqr_n(t, x15, 15); fe_mul(x30, t, x15); // 2^30 - 1
    fe_sqr_n(t, x30, 2); fe_mul(x32, t, x2);   // 2^32 - 1
    // bits 255..224: 32 ones
    // bits 223..192: 0...01
    fe_sqr_n(t, x32, 32); fe_mul(t, t, a);
    // bits 191..96: zeros
    fe_sqr_n(t, t, 96);
    // bits 95..32: 64 ones
    fe_sqr_n(t, t, 32); fe_mul(t, t, x32);
    fe_sqr_n(t, t, 32); fe_mul(t, t, x32);
    // bits 31..0: 30 ones, then 0, 1
    fe_sqr_n(t, t, 30); fe_mul(t, t, x30);
    fe_sqr_n(t, t, 2);  fe_mul(r, t, a);
}

}  // namespace pcmm
