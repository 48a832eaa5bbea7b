// EC-ElGamal decryption (Section 2.4): for a ciphertext (C1, C2) and the
// secret key x, M = C2 - x C1 = m G, and the message m is the discrete
// logarithm of M to base G within a known range [0, mmax] (Section 2.4
// bounds the messages so that this search is feasible).  The logarithm is
// found by baby-step giant-step: with baby steps j G for j in [1, s) kept
// in a hash table keyed on the affine x coordinate, giant steps
// M - g s G (g = 0, 1, ..., floor(mmax / s)) are looked up until one equals
// some j G, giving m = g s + j.  The baby-step table depends on s only (not
// on the key), so one table serves any number of calls.
//
// One thread per ciphertext:
//   x C1 by a left-to-right signed-window (width-4 NAF) double-and-add:
//   the digits of x (recoded once on the host) are the same for every
//   thread, so all branches are warp-uniform; the odd multiples C1, 3 C1,
//   5 C1, 7 C1 are normalised to affine so each non-zero digit costs one
//   mixed addition (about 256 doublings and 51 additions in all);
//   M = C2 + (-x C1), normalised with one inversion per 128-thread block
//   (every normalisation shares its inversion across the block, and the
//   giant-step loop runs until the whole block is done);
//   each giant step probes the table with M's x and confirms a tag match by
//   recomputing j G from the comb table of G (at most 3 mixed additions)
//   and comparing the points exactly, so a tag collision or the point -j G
//   (same x) never gives a wrong answer.
#include <cuda_runtime.h>

#include "comb.cuh"
#include "common.cuh"
#include "profiler.cuh"

using namespace pcmm;

namespace {

constexpr int NAF_MAX = 260;          // digits of a 256-bit scalar in width-4 NAF (<= 257)
constexpr uint32_t BABY_MAX = 1u << 24; // j < 2^24: three 8-bit comb windows
constexpr uint64_t GIANT_MAX = 1u << 20; // giant steps per ciphertext at most

struct Naf {
    int8_t d[NAF_MAX];  // d[i] in {0, +-1, +-3, +-5, +-7}, x = sum d[i] 2^i
    int len;            // d[len - 1] != 0 (len = 0 only for x = 0)
};

__device__ __forceinline__ void fe_neg(fe& r, const fe& a) {
    fe z, t;
    fe_zero(z);
    fe_sub(t, z, a);
    r = t;
}

// Normalise E Jacobian points held in each thread's registers to canonical
// affine coordinates with one field inversion per 128-thread block
// (infinity becomes (0, 0)).  All 128 threads of the block must call.
template <int E>
__device__ __forceinline__ void block_normalize_regs(aff out[E], const jac P[E]) {
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
    fe inv = block4_inverse(acc);
#pragma unroll
    for (int e = E - 1; e >= 0; e--) {
        const fe zinv = e > 0 ? fmul(inv, pref[e - 1]) : inv;
        fe z = P[e].Z;
        const bool is_inf = fe_is_zero(z);
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

// Whether the Jacobian J and the affine A (not infinity) are the same point.
__device__ __forceinline__ bool jac_equals_aff(const jac& J, const aff& A) {
    if (jac_is_inf(J)) return false;
    const fe z2 = fsqr(J.Z);
    const fe z3 = fmul(z2, J.Z);
    return fe_equal(J.X, fmul(A.x, z2)) && fe_equal(J.Y, fmul(A.y, z3));
}

// Slot layout of the baby-step table (cap = 2^k slots of 64 bits, 0 =
// empty): bits 63..32 hold word 1 of the canonical affine x of j G, bits
// 31..0 hold j + 1; the probe sequence starts at word 0 of x modulo cap.
__global__ void __launch_bounds__(128) bsgs_build_kernel(const uint4* __restrict__ gtab, uint32_t s,
                                                         uint32_t mask,
                                                         unsigned long long* __restrict__ slots) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const bool valid = j < s;
    jac R[1];
    comb_mul_u64(R[0], gtab, valid ? j : 1u, 3);
    aff A[1];
    block_normalize_regs<1>(A, R);   // every thread of the block reaches this
    if (!valid) return;
    const unsigned long long val = ((unsigned long long)A[0].x.v[1] << 32) | (unsigned long long)(j + 1);
    uint32_t h = A[0].x.v[0] & mask;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        if (atomicCAS(&slots[h], 0ull, val) == 0ull) break;
        h = (h + 1) & mask;
    }
}

// Odd multiples (2 t + 1) C1, t = 0..3, in affine coordinates (one shared
// inversion per block).  All 128 threads of the block must call.
static __device__ __noinline__ void odd_multiples(aff odd[4], const aff& C1) {
    odd[0] = C1;
    jac D, P[3];
    jac_from_aff(D, C1);
    jac_dbl(D);
    jac_from_aff(P[0], C1);
    jac_add(P[0], D);
    P[1] = P[0];
    jac_add(P[1], D);
    P[2] = P[1];
    jac_add(P[2], D);
    block_normalize_regs<3>(odd + 1, P);
}

// The affine M = C2 - R (R Jacobian) and the giant stride -s G.  All 128
// threads of the block must call.
static __device__ __noinline__ void start_point(aff& M, aff& negS, jac R, const aff& C2,
                                                const uint4* __restrict__ gtab, uint32_t s) {
    fe_neg(R.Y, R.Y);
    jac_madd(R, C2);
    jac J[2];
    J[0] = R;
    comb_mul_u64(J[1], gtab, s, 4);     // s <= 2^24: four comb windows
    aff A[2];
    block_normalize_regs<2>(A, J);
    M = A[0];
    negS = A[1];
    fe_neg(negS.y, negS.y);
}

// Looks M up in the baby-step table; on a confirmed hit j returns true and
// sets *j.
static __device__ __noinline__ bool baby_lookup(const aff& M, const uint4* __restrict__ gtab, uint32_t mask,
                                                const unsigned long long* __restrict__ slots, uint32_t* jout) {
    const uint32_t tag = M.x.v[1];
    uint32_t h = M.x.v[0] & mask;
    for (uint32_t probe = 0; probe <= mask; probe++) {
        const unsigned long long e = slots[h];
        if (e == 0ull) return false;
        if ((uint32_t)(e >> 32) == tag) {
            const uint32_t j = (uint32_t)e - 1u;
            jac J;
            comb_mul_u64(J, gtab, j, 3);
            if (jac_equals_aff(J, M)) {
                *jout = j;
                return true;
            }
        }
        h = (h + 1) & mask;
    }
    return false;
}

// M <- M + Q in affine coordinates (one shared inversion per block).  All
// 128 threads of the block must call.
static __device__ __noinline__ void giant_step(aff& M, const aff& Q) {
    jac J[1];
    jac_from_aff(J[0], M);
    jac_madd(J[0], Q);
    aff A[1];
    block_normalize_regs<1>(A, J);
    M = A[0];
}

// Blocks per SM the register allocation must allow (the scalar
// multiplication is a serial chain per thread: occupancy hides its latency).
#ifndef PCMM_DECRYPT_MINBLOCKS
#define PCMM_DECRYPT_MINBLOCKS 4
#endif

__global__ void __launch_bounds__(128, PCMM_DECRYPT_MINBLOCKS) decrypt_kernel(
        const uint4* __restrict__ gtab, Naf naf, const uint4* __restrict__ ct, size_t count, long long mmax,
        uint32_t s, uint32_t mask, const unsigned long long* __restrict__ slots, long long* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < count;
    const size_t ii = valid ? i : 0;
    aff C1;
    load_aff(C1, ct, count, ii);
    aff odd[4];
    odd_multiples(odd, C1);
    jac R;
    jac_set_inf(R);
    for (int b = naf.len - 1; b >= 0; b--) {
        jac_dbl(R);
        const int d = naf.d[b];
        if (d) {
            aff T = odd[(d < 0 ? -d : d) >> 1];
            if (d < 0 && !aff_is_inf(T)) fe_neg(T.y, T.y);
            jac_madd(R, T);
        }
    }
    aff C2, M, negS;
    load_aff(C2, ct + 4 * count, count, ii);
    start_point(M, negS, R, C2, gtab, s);

    const unsigned long long gmax = (unsigned long long)mmax / s;
    long long found = -1;
    bool done = !valid;
    for (unsigned long long g = 0;; g++) {
        if (!done) {
            uint32_t j = 0;
            if (aff_is_inf(M)) {
                found = (long long)(g * s);
                done = true;
            } else if (baby_lookup(M, gtab, mask, slots, &j)) {
                const unsigned long long v = g * s + j;
                found = v <= (unsigned long long)mmax ? (long long)v : -1;
                done = true;
            }
        }
        if (g >= gmax || group_all(done, true)) break;
        giant_step(M, negS);
    }
    if (valid) out[i] = found;
}

inline unsigned grid_for(size_t count, unsigned block) { return (unsigned)((count + block - 1) / block); }

uint32_t slot_count(uint32_t baby) {
    uint32_t cap = 1;
    while (cap < 2u * baby) cap <<= 1;
    return cap;
}

const uint32_t h_q[8] = {0xfc632551u, 0xf3b9cac2u, 0xa7179e84u, 0xbce6faadu,
                         0xffffffffu, 0xffffffffu, 0x00000000u, 0xffffffffu};

// 1 <= x < q.
bool valid_secret(const uint32_t* x) {
    uint32_t z = 0;
    for (int i = 0; i < 8; i++) z |= x[i];
    if (!z) return false;
    for (int i = 7; i >= 0; i--) {
        if (x[i] < h_q[i]) return true;
        if (x[i] > h_q[i]) return false;
    }
    return false;
}

// Width-4 NAF of x: while x > 0, an odd x gives the digit d = x mods 16
// (in -7..7) and x -= d; then x /= 2.
void naf4(const uint32_t* x32, Naf& naf) {
    uint32_t k[9];
    for (int i = 0; i < 8; i++) k[i] = x32[i];
    k[8] = 0;
    naf.len = 0;
    for (int i = 0; i < NAF_MAX; i++) naf.d[i] = 0;
    for (;;) {
        uint32_t nz = 0;
        for (int i = 0; i < 9; i++) nz |= k[i];
        if (!nz) break;
        int d = 0;
        if (k[0] & 1u) {
            d = (int)(k[0] & 15u);
            if (d >= 8) d -= 16;
            if (d > 0) {
                k[0] -= (uint32_t)d;  // d <= k[0] & 15: no borrow
            } else {
                uint64_t c = (uint64_t)(uint32_t)(-d);
                for (int i = 0; i < 9 && c; i++) {
                    const uint64_t t = (uint64_t)k[i] + c;
                    k[i] = (uint32_t)t;
                    c = t >> 32;
                }
            }
        }
        naf.d[naf.len++] = (int8_t)d;
        for (int i = 0; i < 8; i++) k[i] = (k[i] >> 1) | (k[i + 1] << 31);
        k[8] >>= 1;
    }
}

}  // namespace

extern "C" uint32_t pcmm_bsgs_default_baby(int64_t mmax) {
    if (mmax < 0) return 0;
    uint64_t s = 32;
    while (s < (uint64_t)mmax + 1 && s < BABY_MAX) s <<= 1;
    return (uint32_t)s;
}

extern "C" size_t pcmm_bsgs_bytes(uint32_t baby) {
    if (baby < 1 || baby > BABY_MAX) return 0;
    return (size_t)slot_count(baby) * 8;
}

extern "C" pcmm_status pcmm_bsgs_build(uint32_t baby, void* table, size_t table_bytes, pcmm_stream_t stream) {
    if (baby < 1 || baby > BABY_MAX || !table || ((uintptr_t)table & 15u)) return PCMM_EINVAL;
    const size_t need = pcmm_bsgs_bytes(baby);
    if (table_bytes < need) return PCMM_ENOMEM;
    const uint4* gtab = comb_table_G();
    if (!gtab) return PCMM_EINVAL;
    if (cudaMemsetAsync(table, 0, need, (cudaStream_t)stream) != cudaSuccess) return PCMM_ECUDA;
    if (baby > 1) {
        ProfScope ps(KID_BSGS, (cudaStream_t)stream);
        bsgs_build_kernel<<<grid_for(baby - 1, 128), 128, 0, (cudaStream_t)stream>>>(
            gtab, baby, slot_count(baby) - 1, (unsigned long long*)table);
    }
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_decrypt(const uint32_t* sk_host, const uint32_t* ct, size_t count, int64_t mmax,
                                    uint32_t baby, const void* table, size_t table_bytes, int64_t* out,
                                    pcmm_stream_t stream) {
    if (!sk_host || !ct || !out || !table || mmax < 0 || mmax > ((int64_t)1 << 62)) return PCMM_EINVAL;
    if (baby < 1 || baby > BABY_MAX || ((uintptr_t)table & 15u) || ((uintptr_t)ct & 15u) ||
        ((uintptr_t)out & 7u))
        return PCMM_EINVAL;
    if (!valid_secret(sk_host)) return PCMM_EINVAL;
    if (table_bytes < pcmm_bsgs_bytes(baby)) return PCMM_ENOMEM;
    // Each thread takes up to mmax / baby + 1 giant steps: bound the kernel's length.
    if ((uint64_t)mmax / baby >= GIANT_MAX) return PCMM_EUNSUPPORTED;
    if (count == 0) return PCMM_OK;
    const uint4* gtab = comb_table_G();
    if (!gtab) return PCMM_EINVAL;
    Naf naf;
    naf4(sk_host, naf);
    ProfScope ps(KID_DECRYPT, (cudaStream_t)stream);
    decrypt_kernel<<<grid_for(count, 128), 128, 0, (cudaStream_t)stream>>>(
        gtab, naf, (const uint4*)ct, count, (long long)mmax, baby, slot_count(baby) - 1,
        (const unsigned long long*)table, (long long*)out);
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}
