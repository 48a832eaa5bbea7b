// Group law of NIST P-256, y^2 = x^3 - 3x + b (Sections 2.3 and 4.1), in
// Jacobian coordinates (x = X/Z^2, y = Y/Z^3, infinity has Z = 0) with
// mixed additions against affine points, and the limb-planar point layout
// shared by every kernel.
//
// Formulas (Explicit-Formulas Database names, costs in field mul M and
// squaring S):
//   jac_dbl   "dbl-2001-b" for a = -3          3M + 5S
//   jac_madd  "madd-2007-bl" (Z2 = 1)          7M + 4S
//   jac_add   "add-2007-bl"                    11M + 5S
// All three are made complete: infinity operands, P = Q (doubling) and
// P = -Q (result infinity) are detected and handled on a rare branch.
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

// P <- 2P, a = -3 ("dbl-2001-b").  Infinity (Z = 0) maps to Z3 = 0.
__device__ __forceinline__ void jac_dbl(jac& P) {
    fe delta, gamma, beta, alpha, t0, t1;
    fe_sqr(delta, P.Z);              // delta = Z^2
    fe_sqr(gamma, P.Y);              // gamma = Y^2
    fe_mul(beta, P.X, gamma);        // beta = X gamma
    fe_sub(t0, P.X, delta);
    fe_add(t1, P.X, delta);
    fe_mul(alpha, t0, t1);
    fe_add(t0, alpha, alpha);
    fe_add(alpha, t0, alpha);        // alpha = 3 (X - delta)(X + delta)
    fe_add(t0, P.Y, P.Z);
    fe_sqr(t0, t0);
    fe_sub(t0, t0, gamma);
    fe_sub(P.Z, t0, delta);          // Z3 = (Y + Z)^2 - gamma - delta
    fe_add(beta, beta, beta);
    fe_add(beta, beta, beta);        // 4 beta
    fe_sqr(t0, alpha);
    fe_sub(t0, t0, beta);
    fe_sub(P.X, t0, beta);           // X3 = alpha^2 - 8 beta
    fe_sub(t0, beta, P.X);
    fe_mul(t0, alpha, t0);           // alpha (4 beta - X3)
    fe_sqr(gamma, gamma);
    fe_add(gamma, gamma, gamma);
    fe_add(gamma, gamma, gamma);
    fe_add(gamma, gamma, gamma);     // 8 gamma^2
    fe_sub(P.Y, t0, gamma);          // Y3
}

// P <- P + Q for Jacobian P and affine Q ("madd-2007-bl"), complete.
__device__ __forceinline__ void jac_madd(jac& P, const aff& Q) {
    if (aff_is_inf(Q)) return;
    if (jac_is_inf(P)) {
        P.X = Q.x;
        P.Y = Q.y;
        fe_one(P.Z);
        return;
    }
    fe z1z1, u2, s2, h, hh, i4, j, r, v, t;
    fe_sqr(z1z1, P.Z);               // Z1Z1 = Z1^2
    fe_mul(u2, Q.x, z1z1);           // U2 = X2 Z1Z1
    fe_mul(s2, Q.y, P.Z);
    fe_mul(s2, s2, z1z1);            // S2 = Y2 Z1 Z1Z1
    fe_sub(h, u2, P.X);              // H = U2 - X1
    fe_sub(r, s2, P.Y);
    if (fe_is_zero(h)) {
        if (fe_is_zero(r)) {         // same point: double
            jac_dbl(P);
        } else {                     // opposite points: infinity
            jac_set_inf(P);
        }
        return;
    }
    fe_add(r, r, r);                 // r = 2 (S2 - Y1)
    fe_sqr(hh, h);                   // HH = H^2
    fe_add(i4, hh, hh);
    fe_add(i4, i4, i4);              // I = 4 HH
    fe_mul(j, h, i4);                // J = H I
    fe_mul(v, P.X, i4);              // V = X1 I
    fe_add(t, P.Z, h);
    fe_sqr(t, t);
    fe_sub(t, t, z1z1);
    fe_sub(P.Z, t, hh);              // Z3 = (Z1 + H)^2 - Z1Z1 - HH
    fe_sqr(t, r);
    fe_sub(t, t, j);
    fe_sub(t, t, v);
    fe_sub(P.X, t, v);               // X3 = r^2 - J - 2V
    fe_sub(t, v, P.X);
    fe_mul(t, r, t);                 // r (V - X3)
    fe_mul(j, P.Y, j);
    fe_add(j, j, j);                 // 2 Y1 J
    fe_sub(P.Y, t, j);               // Y3
}

// P <- P + Q, both Jacobian ("add-2007-bl"), complete.
__device__ __forceinline__ void jac_add(jac& P, const jac& Q) {
    if (jac_is_inf(Q)) return;
    if (jac_is_inf(P)) {
        P = Q;
        return;
    }
    fe z1z1, z2z2, u1, u2, s1, s2, h, i, j, r, v, t;
    fe_sqr(z1z1, P.Z);
    fe_sqr(z2z2, Q.Z);
    fe_mul(u1, P.X, z2z2);           // U1 = X1 Z2Z2
    fe_mul(u2, Q.X, z1z1);           // U2 = X2 Z1Z1
    fe_mul(s1, P.Y, Q.Z);
    fe_mul(s1, s1, z2z2);            // S1 = Y1 Z2 Z2Z2
    fe_mul(s2, Q.Y, P.Z);
    fe_mul(s2, s2, z1z1);            // S2 = Y2 Z1 Z1Z1
    fe_sub(h, u2, u1);               // H = U2 - U1
    fe_sub(r, s2, s1);
    if (fe_is_zero(h)) {
        if (fe_is_zero(r)) {
            jac_dbl(P);
        } else {
            jac_set_inf(P);
        }
        return;
    }
    fe_add(r, r, r);                 // r = 2 (S2 - S1)
    fe_add(i, h, h);
    fe_sqr(i, i);                    // I = (2H)^2
    fe_mul(j, h, i);                 // J = H I
    fe_mul(v, u1, i);                // V = U1 I
    fe_add(t, P.Z, Q.Z);
    fe_sqr(t, t);
    fe_sub(t, t, z1z1);
    fe_sub(t, t, z2z2);
    fe_mul(P.Z, t, h);               // Z3 = ((Z1 + Z2)^2 - Z1Z1 - Z2Z2) H
    fe_sqr(t, r);
    fe_sub(t, t, j);
    fe_sub(t, t, v);
    fe_sub(P.X, t, v);               // X3 = r^2 - J - 2V
    fe_sub(t, v, P.X);
    fe_mul(t, r, t);
    fe_mul(s1, s1, j);
    fe_add(s1, s1, s1);              // 2 S1 J
    fe_sub(P.Y, t, s1);              // Y3
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
    fe z2, z3;
    fe_sqr(z2, zinv);
    fe_mul(z3, z2, zinv);
    fe_mul(Q.x, P.X, z2);
    fe_mul(Q.y, P.Y, z3);
    fe_canon(Q.x, Q.x);
    fe_canon(Q.y, Q.y);
}

}  // namespace pcmm
