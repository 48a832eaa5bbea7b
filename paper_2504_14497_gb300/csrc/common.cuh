// Helpers shared by the PC-MM kernels: status codes, warp-level batched
// affine normalisation (Montgomery's simultaneous-inversion trick with
// warp-shuffle prefix products), and the lane-planar scratch layout.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pcmm.h"
#include "ec.cuh"

namespace pcmm {

// Error bits a kernel may raise in a device status word.
enum : uint32_t {
    DEV_ERR_A_RANGE = 1u << 0,  // an entry of A is >= 2^w
    DEV_ERR_PLAN = 1u << 1,     // a plan size exceeded its bound
    DEV_ERR_TIMEOUT = 1u << 2,  // a bounded device-side wait gave up
};

// Waits until *ctr >= target, polling with short sleeps, for at most about
// 2^22 polls (roughly a second).  Gives up early when another warp has
// already raised DEV_ERR_TIMEOUT in *status; raises it itself when the bound
// runs out.  Returns whether the target was reached.  Call from one lane.
__device__ __forceinline__ bool wait_at_least(const int* ctr, int target, uint32_t* status) {
    for (int it = 0; it < (1 << 22); it++) {
        if (*(volatile const int*)ctr >= target) {
            __threadfence();
            return true;
        }
        if (*(volatile const uint32_t*)status & DEV_ERR_TIMEOUT) return false;
        __nanosleep(256);
    }
    atomicOr(status, DEV_ERR_TIMEOUT);
    return false;
}

__device__ __forceinline__ fe fe_shfl_up(const fe& a, unsigned d) {
    fe r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = __shfl_up_sync(0xffffffffu, a.v[i], d);
    return r;
}

__device__ __forceinline__ fe fe_shfl_down(const fe& a, unsigned d) {
    fe r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = __shfl_down_sync(0xffffffffu, a.v[i], d);
    return r;
}

__device__ __forceinline__ fe fe_shfl(const fe& a, int src) {
    fe r;
#pragma unroll
    for (int i = 0; i < 8; i++) r.v[i] = __shfl_sync(0xffffffffu, a.v[i], src);
    return r;
}

// Given each lane's value t (non-zero), returns t^-1 using one field
// inversion for the whole warp: inclusive prefix and suffix products over
// the lanes by shuffles, the inverse of the warp total, and
// t^-1 = total^-1 * (product of the other lanes).  All 32 lanes must call.
__device__ __forceinline__ void warp_inverse(fe& tinv, const fe& t) {
    const unsigned lane = threadIdx.x & 31u;
    fe pre = t, suf = t, o;
#pragma unroll
    for (unsigned d = 1; d < 32; d <<= 1) {
        o = fe_shfl_up(pre, d);
        if (lane >= d) pre = fmul(pre, o);
    }
#pragma unroll
    for (unsigned d = 1; d < 32; d <<= 1) {
        o = fe_shfl_down(suf, d);
        if (lane + d < 32u) suf = fmul(suf, o);
    }
    fe total = fe_shfl(pre, 31);
    fe pex = fe_shfl_up(pre, 1);    // product of lanes below
    fe sex = fe_shfl_down(suf, 1);  // product of lanes above
    if (lane == 0) fe_one(pex);
    if (lane == 31) fe_one(sex);
    fe inv;
    fe_inv(inv, total);
    inv = fmul(inv, pex);
    tinv = fmul(inv, sex);
}

// Normalise E Jacobian points held in each lane's registers to canonical
// affine coordinates; infinity (Z = 0) becomes (0, 0).  One inversion per
// warp for 32 * E points.  All 32 lanes must call.
template <int E>
__device__ __forceinline__ void warp_normalize_regs(aff out[E], const jac P[E]) {
    fe pref[E];
    fe acc;
    fe_one(acc);
#pragma unroll
    for (int e = 0; e < E; e++) {
        fe z = P[e].Z;
        if (fe_is_zero(z)) fe_one(z);
        acc = fmul(acc, z);
        pref[e] = acc;
    }
    fe inv;
    warp_inverse(inv, acc);
#pragma unroll
    for (int e = E - 1; e >= 0; e--) {
        fe zinv;
        if (e > 0) zinv = fmul(inv, pref[e - 1]);
        else zinv = inv;
        fe z = P[e].Z;
        bool is_inf = fe_is_zero(z);
        if (is_inf) fe_one(z);
        inv = fmul(inv, z);
        if (is_inf) {
            fe_zero(out[e].x);
            fe_zero(out[e].y);
        } else {
            jac_to_aff_with_zinv(out[e], P[e], zinv);
        }
    }
}

// ---------------------------------------------------------------------------
// Lane-planar scratch: a per-warp array of E entries, each entry holding Q
// quads for each of the 32 lanes; quad q of entry e for lane L lives at
// uint4 index (e * Q + q) * 32 + L, so every access is a coalesced 512-byte
// warp transaction.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void lp_store_jac(uint4* base, int e, unsigned lane, const jac& P) {
    uint4* b = base + (size_t)e * 6 * 32 + lane;
    b[0] = fe_lo(P.X);
    b[32] = fe_hi(P.X);
    b[64] = fe_lo(P.Y);
    b[96] = fe_hi(P.Y);
    b[128] = fe_lo(P.Z);
    b[160] = fe_hi(P.Z);
}

__device__ __forceinline__ void lp_load_jac(jac& P, const uint4* base, int e, unsigned lane) {
    const uint4* b = base + (size_t)e * 6 * 32 + lane;
    fe_from_quads(P.X, b[0], b[32]);
    fe_from_quads(P.Y, b[64], b[96]);
    fe_from_quads(P.Z, b[128], b[160]);
}

__device__ __forceinline__ void lp_load_z(fe& z, const uint4* base, int e, unsigned lane) {
    const uint4* b = base + (size_t)e * 6 * 32 + lane;
    fe_from_quads(z, b[128], b[160]);
}

__device__ __forceinline__ void lp_store_fe(uint4* base, int e, unsigned lane, const fe& a) {
    uint4* b = base + (size_t)e * 2 * 32 + lane;
    b[0] = fe_lo(a);
    b[32] = fe_hi(a);
}

__device__ __forceinline__ void lp_load_fe(fe& a, const uint4* base, int e, unsigned lane) {
    const uint4* b = base + (size_t)e * 2 * 32 + lane;
    fe_from_quads(a, b[0], b[32]);
}

}  // namespace pcmm

#define PCMM_CUDA_CHECK_LAUNCH()                                   \
    do {                                                           \
        cudaError_t _e = cudaGetLastError();                       \
        if (_e != cudaSuccess) return PCMM_ECUDA;                  \
    } while (0)
