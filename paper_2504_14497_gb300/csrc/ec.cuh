// Group law of NIST P-256, y^2 = x^3 - 3x + b (Sections 2.3 and 4.1), in
// Jacobian coordinates (x = X/Z^2, y = Y/Z^3, infinity has Z = 0) with
// mixed additions against affine points, and the limb-planar point layout
// shared by every kernel.
//
// Formulas (costs in field multiplications M and squarings S):
//   jac_dbl   doubling for a = -3 ("dbl-2001-b" in the Explicit-Formulas
//             Database)                                         3M + 5S
//   jac_madd  textbook mixed addition: U2 = x2 Z1^2, S2 = y2 Z1^3,
//             H = U2 - X1, R = S2 - Y1, X3 = R^2 - H^3 - 2 X1 H^2,
//             Y3 = R (X1 H^2 - X3) - Y1 H^3, Z3 = Z1 H          8M + 3S
//   jac_add   the same with U1 = X1 Z2^2, S1 = Y1 Z2^3,
//             Z3 = Z1 Z2 H                                      12M + 4S
// Y3 in both additions is a difference of two products reduced once
// (fmulsub).  These formulas need fewer additions and subtractions than the
// 7M + 4S / 11M + 5S variants, and additions, not multiplications, bound
// this code on sm_103a.  All three are complete: infinity operands, P = Q
// (doubling) and P = -Q (result infinity) are detected and handled on a rare
// branch.
//
// Point arrays in global memory are QUAD-PLANAR: an array of N points stores
// coordinate quad q (4 consecutive 32-bit limbs) of point i at uint4 index
// q * N + i.  Affine points have 4 quads (x lo, x hi, y lo, y hi), Jacobian
// points 6 (X lo, X hi, Y lo, Y hi, Z lo, Z hi).  Adjacent threads reading
// adjacent points therefore issue fully coalesced 16-byte loads.  The affine
// point at infinity is encoded as x = y = 0, which is not on the curve.
#pragma once
#include "fp256.cuh"

namespace pcmm {

struct aff {
    fe x, y;
};
struct jac {
    fe X, Y, Z;
};

__device__ __forceinline__ void jac_set_inf(jac& P) {
    fe_one(P.X);
    fe_one(P.Y);
    fe_zero(P.Z);
}

__device__ __forceinline__ bool jac_is_inf(const jac& P) { return fe_is_zero(P.Z); }

__device__ __forceinline__ bool aff_is_inf(const aff& Q) {
    uint32_t z = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) z |= Q.x.v[i] | Q.y.v[i];
    return z == 0u;
}

__device__ __forceinline__ void jac_from_aff(jac& P, const aff& Q) {
    if (aff_is_inf(Q)) {
        jac_set_inf(P);
        return;
    }
    P.X = Q.x;
    P.Y = Q.y;
    fe_one(P.Z);
}

// P <- 2P, a = -3: delta = Z^2, gamma = Y^2, beta = X gamma,
// alpha = 3 (X - delta)(X + delta), X3 = alpha^2 - 8 beta,
// Z3 = (Y + Z)^2 - gamma - delta, Y3 = alpha (4 beta - X3) - 8 gamma^2.
// Infinity (Z = 0) maps to Z3 = 0.
__device__ __forceinline__ void jac_dbl(jac& P) {
    fe delta, gamma, beta, alpha, t0, t1;
    delta = fsqr(P.Z);
    gamma = fsqr(P.Y);
    beta = fmul(P.X, gamma);
    fe_sub(t0, P.X, delta);
    fe_add(t1, P.X, delta);
    alpha = fmul(t0, t1);
    fe_add(t0, alpha, alpha);
    fe_add(alpha, t0, alpha);        // alpha = 3 (X - delta)(X + delta)
    fe_add(t0, P.Y, P.Z);
    t0 = fsqr(t0);
    fe_sub(t0, t0, gamma);
    fe_sub(P.Z, t0, delta);          // Z3
    fe_add(beta, beta, beta);
    fe_add(beta, beta, beta);        // 4 beta
    t0 = fsqr(alpha);
    fe_sub(t0, t0, beta);
    fe_sub(P.X, t0, beta);           // X3 = alpha^2 - 8 beta
    fe_sub(t0, beta, P.X);
    t0 = fmul(alpha, t0);            // alpha (4 beta - X3)
    gamma = fsqr(gamma);
    fe_add(gamma, gamma, gamma);
    fe_add(gamma, gamma, gamma);
    fe_add(gamma, gamma, gamma);     // 8 gamma^2
    fe_sub(P.Y, t0, gamma);          // Y3
}

// P <- P + Q for Jacobian P and affine Q, complete.
__device__ __forceinline__ void jac_madd(jac& P, const aff& Q) {
    if (aff_is_inf(Q)) return;
    if (jac_is_inf(P)) {
        P.X = Q.x;
        P.Y = Q.y;
        fe_one(P.Z);
        return;
    }
    fe t1, t2, t3, t4, x3;
    t1 = fsqr(P.Z);                  // Z1^2
    t2 = fmul(t1, P.Z);              // Z1^3
    t1 = fmul(t1, Q.x);              // U2
    t2 = fmul(t2, Q.y);              // S2
    fe_sub(t1, t1, P.X);             // H
    fe_sub(t2, t2, P.Y);             // R
    if (fe_is_zero(t1)) {
        if (fe_is_zero(t2)) jac_dbl(P);   // same point
        else jac_set_inf(P);              // opposite points
        return;
    }
    P.Z = fmul(P.Z, t1);             // Z3 = Z1 H
    t4 = fsqr(t1);                   // H^2
    t3 = fmul(t4, t1);               // H^3
    t4 = fmul(t4, P.X);              // X1 H^2
    fe_add(t1, t4, t4);              // 2 X1 H^2
    x3 = fsqr(t2);                   // R^2
    fe_sub(x3, x3, t1);
    fe_sub(x3, x3, t3);              // X3 = R^2 - 2 X1 H^2 - H^3
    fe_sub(t4, t4, x3);              // X1 H^2 - X3
    P.Y = fmulsub(t4, t2, t3, P.Y);  // Y3 = R (X1 H^2 - X3) - Y1 H^3
    P.X = x3;
}

// Accumulator of a long run of mixed additions in which Z is never needed
// itself: (X, Y, ZZ, ZZZ) with ZZ = Z^2 and ZZZ = Z^3 of some Jacobian Z
// (infinity: ZZ = ZZZ = 0).  A mixed addition then updates ZZ and ZZZ with
// the H^2 and H^3 it computes anyway (8M + 2S instead of 8M + 3S).
struct jacz {
    fe X, Y, ZZ, ZZZ;
};

__device__ __forceinline__ void jacz_set_inf(jacz& P) {
    fe_one(P.X);
    fe_one(P.Y);
    fe_zero(P.ZZ);
    fe_zero(P.ZZZ);
}

__device__ __forceinline__ void jacz_from_jac(jacz& R, const jac& P) {
    R.X = P.X;
    R.Y = P.Y;
    R.ZZ = fsqr(P.Z);
    R.ZZZ = fmul(R.ZZ, P.Z);
}

// Jacobian representative without an inversion: with Z' = ZZ ZZZ = Z^5,
// X' = x Z'^2 = X ZZ^4 and Y' = y Z'^3 = Y ZZZ^4 (4S + 3M).  Infinity maps
// to Z' = 0.  An accumulator that only ever copied one affine point (ZZ and
// ZZZ both exactly 1) is returned as it is.
__device__ __forceinline__ void jac_from_jacz(jac& R, const jacz& P) {
    if (fe_is_one(P.ZZ) && fe_is_one(P.ZZZ)) {
        R.X = P.X;
        R.Y = P.Y;
        R.Z = P.ZZ;
        return;
    }
    fe t = fsqr(P.ZZ);
    t = fsqr(t);
    R.X = fmul(P.X, t);
    t = fsqr(P.ZZZ);
    t = fsqr(t);
    R.Y = fmul(P.Y, t);
    R.Z = fmul(P.ZZ, P.ZZZ);
}

// INL: which field operations are inlined (bit 0 the squarings, bit 1 the
// fused a b - c d, bit 2 U2 and S2, bit 3 H^3 and the ZZ, ZZZ updates,
// bit 4 X1 H^2); the rest run out of line.
template <int INL>
__device__ __forceinline__ void jacz_madd_t(jacz& P, const aff& Q) {
    constexpr bool IS = (INL & 1) != 0, IF = (INL & 2) != 0, IU = (INL & 4) != 0, IZ = (INL & 8) != 0,
                   IX = (INL & 16) != 0;
    if (aff_is_inf(Q)) return;
    if (fe_is_zero(P.ZZ)) {
        P.X = Q.x;
        P.Y = Q.y;
        fe_one(P.ZZ);
        fe_one(P.ZZZ);
        return;
    }
    fe t1, t2, t3, t4, x3;
    t1 = mul_t<IU>(P.ZZ, Q.x);            // U2
    t2 = mul_t<IU>(P.ZZZ, Q.y);           // S2
    fe_sub(t1, t1, P.X);             // H
    fe_sub(t2, t2, P.Y);             // R
    if (fe_is_zero(t1)) {
        if (fe_is_zero(t2)) {        // P = Q: the result is 2Q, from Q's affine coordinates
            jac D;
            jac_from_aff(D, Q);
            jac_dbl(D);
            jacz_from_jac(P, D);
        } else {                     // P = -Q
            jacz_set_inf(P);
        }
        return;
    }
    t4 = sqr_t<IS>(t1);                   // H^2
    t3 = mul_t<IZ>(t4, t1);               // H^3
    P.ZZ = mul_t<IZ>(P.ZZ, t4);           // ZZ3 = ZZ1 H^2
    P.ZZZ = mul_t<IZ>(P.ZZZ, t3);         // ZZZ3 = ZZZ1 H^3
    t4 = mul_t<IX>(t4, P.X);              // X1 H^2
    fe_add(t1, t4, t4);              // 2 X1 H^2
    x3 = sqr_t<IS>(t2);                   // R^2
    fe_sub(x3, x3, t1);
    fe_sub(x3, x3, t3);              // X3 = R^2 - 2 X1 H^2 - H^3
    fe_sub(t4, t4, x3);              // X1 H^2 - X3
    P.Y = mulsub_t<IF>(t4, t2, t3, P.Y);  // Y3 = R (X1 H^2 - X3) - Y1 H^3
    P.X = x3;
}

__device__ __forceinline__ void jacz_madd(jacz& P, const aff& Q) { jacz_madd_t<0>(P, Q); }

// Doubling in (X, Y, ZZ, ZZZ) coordinates (dbl-2001-b with delta = ZZ): Z
// would become 2 Y Z, so ZZ is multiplied by rr2 = 4 Y^2 and ZZZ by
// rr3 = 8 Y^3; both factors are returned.
__device__ __forceinline__ void jacz_dbl_ratio(jacz& P, fe& rr2, fe& rr3) {
    fe gamma, beta, alpha, t0, t1;
    gamma = fsqr(P.Y);
    beta = fmul(P.X, gamma);
    fe_sub(t0, P.X, P.ZZ);
    fe_add(t1, P.X, P.ZZ);
    alpha = fmul(t0, t1);
    fe_add(t0, alpha, alpha);
    fe_add(alpha, t0, alpha);        // alpha = 3 (X - ZZ)(X + ZZ)
    fe_add(beta, beta, beta);
    fe_add(beta, beta, beta);        // 4 beta
    fe_add(rr2, gamma, gamma);
    fe_add(rr2, rr2, rr2);           // 4 Y^2
    t1 = fmul(P.Y, gamma);           // Y^3
    fe_add(rr3, t1, t1);
    fe_add(rr3, rr3, rr3);
    fe_add(rr3, rr3, rr3);           // 8 Y^3
    t0 = fsqr(alpha);
    fe_sub(t0, t0, beta);
    fe_sub(P.X, t0, beta);           // X3 = alpha^2 - 8 beta
    fe_sub(t0, beta, P.X);
    t0 = fmul(alpha, t0);            // alpha (4 beta - X3)
    gamma = fsqr(gamma);
    fe_add(gamma, gamma, gamma);
    fe_add(gamma, gamma, gamma);
    fe_add(gamma, gamma, gamma);     // 8 Y^4
    fe_sub(P.Y, t0, gamma);          // Y3
    P.ZZ = fmul(P.ZZ, rr2);
    P.ZZZ = fmul(P.ZZZ, rr3);
}

// jacz_madd for a chain normalised by walking ZZ^-1 and ZZZ^-1 backwards:
// also returns the factors rr2, rr3 that ZZ and ZZZ were multiplied by (H^2
// and H^3 for an addition; for a doubling those of jacz_dbl_ratio; 1 when
// Q is infinity; for the first step, from infinity, ZZ = ZZZ = 1 and the
// factors are 1).  ok is cleared when no such factors exist (infinity
// after the first step, or a result at infinity).
// INL as for jacz_madd_t (bit 0 squarings, bit 1 the fused a b - c d).
template <int INL>
__device__ __forceinline__ void jacz_madd_ratio_t(jacz& P, const aff& Q, fe& rr2, fe& rr3, bool& ok, bool first) {
    constexpr bool IS = (INL & 1) != 0, IF = (INL & 2) != 0;
    fe_one(rr2);
    fe_one(rr3);
    if (aff_is_inf(Q)) {
        if (fe_is_zero(P.ZZ)) ok = false;
        return;
    }
    if (fe_is_zero(P.ZZ)) {
        P.X = Q.x;
        P.Y = Q.y;
        fe_one(P.ZZ);
        fe_one(P.ZZZ);
        if (!first) ok = false;
        return;
    }
    fe t1, t2, t3, t4, x3;
    t1 = fmul(P.ZZ, Q.x);            // U2
    t2 = fmul(P.ZZZ, Q.y);           // S2
    fe_sub(t1, t1, P.X);             // H
    fe_sub(t2, t2, P.Y);             // R
    if (fe_is_zero(t1)) {
        if (fe_is_zero(t2)) {        // same point
            jacz_dbl_ratio(P, rr2, rr3);
            if (fe_is_zero(rr2) || fe_is_zero(P.ZZ)) ok = false;
        } else {                     // opposite points
            jacz_set_inf(P);
            ok = false;
        }
        return;
    }
    t4 = sqr_t<IS>(t1);              // H^2
    t3 = fmul(t4, t1);               // H^3
    rr2 = t4;
    rr3 = t3;
    P.ZZ = fmul(P.ZZ, t4);
    P.ZZZ = fmul(P.ZZZ, t3);
    t4 = fmul(t4, P.X);              // X1 H^2
    fe_add(t1, t4, t4);              // 2 X1 H^2
    x3 = sqr_t<IS>(t2);              // R^2
    fe_sub(x3, x3, t1);
    fe_sub(x3, x3, t3);              // X3 = R^2 - 2 X1 H^2 - H^3
    fe_sub(t4, t4, x3);              // X1 H^2 - X3
    P.Y = mulsub_t<IF>(t4, t2, t3, P.Y);  // Y3 = R (X1 H^2 - X3) - Y1 H^3
    P.X = x3;
}

// P <- P + Q, both Jacobian, complete.
__device__ __forceinline__ void jac_add(jac& P, const jac& Q) {
    if (jac_is_inf(Q)) return;
    if (jac_is_inf(P)) {
        P = Q;
        return;
    }
    fe z1z1, z2z2, u1, u2, s1, s2, h, r, t3, t4, x3;
    z1z1 = fsqr(P.Z);
    z2z2 = fsqr(Q.Z);
    u1 = fmul(P.X, z2z2);            // U1 = X1 Z2^2
    u2 = fmul(Q.X, z1z1);            // U2 = X2 Z1^2
    s1 = fmul(P.Y, fmul(z2z2, Q.Z)); // S1 = Y1 Z2^3
    s2 = fmul(Q.Y, fmul(z1z1, P.Z)); // S2 = Y2 Z1^3
    fe_sub(h, u2, u1);               // H
    fe_sub(r, s2, s1);               // R
    if (fe_is_zero(h)) {
        if (fe_is_zero(r)) jac_dbl(P);
        else jac_set_inf(P);
        return;
    }
    P.Z = fmul(fmul(P.Z, Q.Z), h);   // Z3 = Z1 Z2 H
    t4 = fsqr(h);                    // H^2
    t3 = fmul(t4, h);                // H^3
    t4 = fmul(t4, u1);               // U1 H^2
    fe_add(u2, t4, t4);              // 2 U1 H^2
    x3 = fsqr(r);
    fe_sub(x3, x3, u2);
    fe_sub(x3, x3, t3);              // X3 = R^2 - 2 U1 H^2 - H^3
    fe_sub(t4, t4, x3);              // U1 H^2 - X3
    P.Y = fmulsub(t4, r, t3, s1);    // Y3 = R (U1 H^2 - X3) - S1 H^3
    P.X = x3;
}

// P <- k P for a small non-negative scalar k (at most 32 bits) by
// left-to-right double-and-add over the bits below the leading one.
__device__ __forceinline__ void jac_mul_small(jac& R, const aff& P, uint32_t k) {
    jac_set_inf(R);
    if (k == 0u || aff_is_inf(P)) return;
    int top = 31 - __clz(k);
    jac_from_aff(R, P);
    for (int b = top - 1; b >= 0; b--) {
        jac_dbl(R);
        if ((k >> b) & 1u) jac_madd(R, P);
    }
}

// ---------------------------------------------------------------------------
// Quad-planar loads and stores.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void fe_from_quads(fe& a, uint4 lo, uint4 hi) {
    a.v[0] = lo.x; a.v[1] = lo.y; a.v[2] = lo.z; a.v[3] = lo.w;
    a.v[4] = hi.x; a.v[5] = hi.y; a.v[6] = hi.z; a.v[7] = hi.w;
}

__device__ __forceinline__ uint4 fe_lo(const fe& a) { return make_uint4(a.v[0], a.v[1], a.v[2], a.v[3]); }
__device__ __forceinline__ uint4 fe_hi(const fe& a) { return make_uint4(a.v[4], a.v[5], a.v[6], a.v[7]); }

__device__ __forceinline__ void load_aff(aff& Q, const uint4* __restrict__ base, size_t stride, size_t i) {
    uint4 q0 = base[i], q1 = base[stride + i], q2 = base[2 * stride + i], q3 = base[3 * stride + i];
    fe_from_quads(Q.x, q0, q1);
    fe_from_quads(Q.y, q2, q3);
}

// L2-only loads (ld.global.cg), for data written by other SMs during the
// same kernel launch.
__device__ __forceinline__ void load_aff_cg(aff& Q, const uint4* __restrict__ base, size_t stride, size_t i) {
    uint4 q0 = __ldcg(base + i), q1 = __ldcg(base + stride + i), q2 = __ldcg(base + 2 * stride + i),
          q3 = __ldcg(base + 3 * stride + i);
    fe_from_quads(Q.x, q0, q1);
    fe_from_quads(Q.y, q2, q3);
}

__device__ __forceinline__ void load_jac_cg(jac& P, const uint4* __restrict__ base, size_t stride, size_t i) {
    uint4 q0 = __ldcg(base + i), q1 = __ldcg(base + stride + i), q2 = __ldcg(base + 2 * stride + i);
    uint4 q3 = __ldcg(base + 3 * stride + i), q4 = __ldcg(base + 4 * stride + i),
          q5 = __ldcg(base + 5 * stride + i);
    fe_from_quads(P.X, q0, q1);
    fe_from_quads(P.Y, q2, q3);
    fe_from_quads(P.Z, q4, q5);
}

__device__ __forceinline__ void store_aff(uint4* __restrict__ base, size_t stride, size_t i, const aff& Q) {
    base[i] = fe_lo(Q.x);
    base[stride + i] = fe_hi(Q.x);
    base[2 * stride + i] = fe_lo(Q.y);
    base[3 * stride + i] = fe_hi(Q.y);
}

__device__ __forceinline__ void load_jac(jac& P, const uint4* __restrict__ base, size_t stride, size_t i) {
    uint4 q0 = base[i], q1 = base[stride + i], q2 = base[2 * stride + i];
    uint4 q3 = base[3 * stride + i], q4 = base[4 * stride + i], q5 = base[5 * stride + i];
    fe_from_quads(P.X, q0, q1);
    fe_from_quads(P.Y, q2, q3);
    fe_from_quads(P.Z, q4, q5);
}

__device__ __forceinline__ void store_jac(uint4* __restrict__ base, size_t stride, size_t i, const jac& P) {
    base[i] = fe_lo(P.X);
    base[stride + i] = fe_hi(P.X);
    base[2 * stride + i] = fe_lo(P.Y);
    base[3 * stride + i] = fe_hi(P.Y);
    base[4 * stride + i] = fe_lo(P.Z);
    base[5 * stride + i] = fe_hi(P.Z);
}

__device__ __forceinline__ void load_fe(fe& a, const uint4* __restrict__ base, size_t stride, size_t i) {
    fe_from_quads(a, base[i], base[stride + i]);
}

__device__ __forceinline__ void store_fe(uint4* __restrict__ base, size_t stride, size_t i, const fe& a) {
    base[i] = fe_lo(a);
    base[stride + i] = fe_hi(a);
}

// Affine from Jacobian given zinv = Z^-1 (Z != 0); canonical output.
__device__ __forceinline__ void jac_to_aff_with_zinv(aff& Q, const jac& P, const fe& zinv) {
    fe z2 = fsqr(zinv);
    fe z3 = fmul(z2, zinv);
    Q.x = fmul(P.X, z2);
    Q.y = fmul(P.Y, z3);
    fe_canon(Q.x, Q.x);
    fe_canon(Q.y, Q.y);
}

}  // namespace pcmm
