// Helpers shared by the PC-MM kernels: status codes, the bounded device
// wait, batched inversion (Montgomery's simultaneous-inversion trick with
// warp-shuffle prefix products, optionally shared by the four warps of a
// block), warp-level affine normalisation, and the lane-planar scratch
// layout.
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
    DEV_ERR_BOUNDS = 1u << 3,   // a plan index outside its table (PCMM_DEBUG_BOUNDS builds)
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

// warp_inverse with one field inversion shared by the four warps of a
// 128-thread block (the inversion, executed by every lane of a warp, costs
// as much as about 250 multiplications): each warp's total goes to shared
// memory, warp 0 inverts the product of the four and hands each warp the
// inverse of its total.  All 128 threads of the block must call, in the same
// order as every other block-level call (blockDim.x must be 128).
static __device__ __noinline__ fe block4_inverse(fe t) {
    __shared__ fe sh_tot[4];
    __shared__ fe sh_inv[4];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
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
    fe pex = fe_shfl_up(pre, 1);
    fe sex = fe_shfl_down(suf, 1);
    if (lane == 0) fe_one(pex);
    if (lane == 31) fe_one(sex);
    if (lane == 0) sh_tot[warp] = total;
    __syncthreads();
    if (warp == 0) {
        const fe p01 = fmul(sh_tot[0], sh_tot[1]);
        const fe p012 = fmul(p01, sh_tot[2]);
        fe i;
        fe_inv(i, fmul(p012, sh_tot[3]));
        const fe i3 = fmul(i, p012);                 // total_3^-1
        const fe i012 = fmul(i, sh_tot[3]);          // (t0 t1 t2)^-1
        const fe i2 = fmul(i012, p01);               // total_2^-1
        const fe i01 = fmul(i012, sh_tot[2]);        // (t0 t1)^-1
        const fe i1 = fmul(i01, sh_tot[0]);
        const fe i0 = fmul(i01, sh_tot[1]);
        if (lane == 0) {
            sh_inv[0] = i0;
            sh_inv[1] = i1;
            sh_inv[2] = i2;
            sh_inv[3] = i3;
        }
    }
    __syncthreads();
    fe inv = sh_inv[warp];
    inv = fmul(inv, pex);
    return fmul(inv, sex);
}

// t^-1 per lane: block4_inverse when `shared` (then all 128 threads of the
// block must call), warp_inverse otherwise.
__device__ __forceinline__ void group_inverse(fe& tinv, const fe& t, bool shared) {
    if (shared) tinv = block4_inverse(t);
    else warp_inverse(tinv, t);
}

// Whether x holds on every lane of the warp or, with `shared`, on every
// thread of the block (then all threads of the block must call).
__device__ __forceinline__ bool group_all(bool x, bool shared) {
    return shared ? __syncthreads_and(x) != 0 : __all_sync(0xffffffffu, x);
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
