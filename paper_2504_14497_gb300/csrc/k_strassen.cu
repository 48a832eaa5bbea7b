// Strassen PC-MM (Section 3.1): A (plaintext) times Enc(B) by recursive
// 2 x 2 block partitioning with seven block products per step,
//   M1 = (A11 + A22)(B11 + B22)   M2 = (A21 + A22) B11
//   M3 = A11 (B12 - B22)          M4 = A22 (B21 - B11)
//   M5 = (A11 + A12) B22          M6 = (A21 - A11)(B11 + B12)
//   M7 = (A12 - A22)(B21 + B22)
//   C11 = M1 + M4 - M5 + M7, C12 = M3 + M5, C21 = M2 + M4,
//   C22 = M1 - M2 + M3 + M6,
// the plaintext block sums being integer additions and the ciphertext ones
// point additions (5 + 8 = 13 per step), and the schoolbook product at the
// leaves.  The paper's second comparison system, beside Cussen's method.
//
// GB300 design: breadth first.  Level t of the recursion holds 7^t nodes,
// each a plaintext block (int16: the block sums widen by one bit per level
// and take both signs) and an affine ciphertext block, stored node after
// node in one array per level.  Each level down is two launches over all of
// its nodes (plaintext sums; ciphertext sums normalised to affine, one warp
// inversion per 64 points), the 7^d leaf products are one launch of a signed
// schoolbook kernel, and each level up is one launch that assembles every
// parent's four quadrants from its seven children by full Jacobian
// additions.  Nothing is recursive on the device.
#include <cuda_runtime.h>

#include "common.cuh"
#include "profiler.cuh"

using namespace pcmm;

namespace {

constexpr int STRASSEN_MAX_LEVELS = 7;

// Plaintext block sums of one recursion step: for every parent node q and
// position (i, k) of its top-left quadrant, the seven children's entries
// (TS: int16, or int32 when w + levels > 15).  The top level (TOP) reads A
// (uint8 or uint16, entries masked to w bits, out-of-range entries flagged
// in the status word); deeper levels read the parent level's sums.
template <class TIN, class TS, bool TOP>
__global__ void __launch_bounds__(128) strassen_psum_kernel(const TIN* __restrict__ P, int mp, int np,
                                                            long long nodes, uint32_t amask,
                                                            TS* __restrict__ S, uint32_t* status) {
    const int mh = mp / 2, nh = np / 2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nodes * mh * nh) return;
    const int k = (int)(t % nh);
    const int i = (int)((t / nh) % mh);
    const long long q = t / ((long long)nh * mh);
    const TIN* b = P + (size_t)q * mp * np;
    int a[4];
    const size_t idx[4] = {(size_t)i * np + k, (size_t)i * np + nh + k, (size_t)(mh + i) * np + k,
                           (size_t)(mh + i) * np + nh + k};
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const TIN v = b[idx[u]];
        if (TOP) {
            if ((uint32_t)v & ~amask) atomicOr(status, DEV_ERR_A_RANGE);
            a[u] = (int)((uint32_t)v & amask);
        } else {
            a[u] = (int)v;
        }
    }
    const int a11 = a[0], a12 = a[1], a21 = a[2], a22 = a[3];
    const size_t st = (size_t)mh * nh;
    TS* s = S + (size_t)7 * q * st + (size_t)i * nh + k;
    s[0 * st] = (TS)(a11 + a22);
    s[1 * st] = (TS)(a21 + a22);
    s[2 * st] = (TS)a11;
    s[3 * st] = (TS)a22;
    s[4 * st] = (TS)(a11 + a12);
    s[5 * st] = (TS)(a21 - a11);
    s[6 * st] = (TS)(a12 - a22);
}

// -Q for an affine point (infinity stays (0, 0)).
__device__ __forceinline__ void aff_negate(aff& Q) {
    if (aff_is_inf(Q)) return;
    fe z;
    fe_zero(z);
    fe_sub(Q.y, z, Q.y);
}

// Ciphertext block sums of one recursion step: for every parent node q and
// position (k, j) of its top-left quadrant, the seven children's
// ciphertexts, both points: copies B11 (child 2) and B22 (child 5), and
// B11 + B22, B12 - B22, B21 - B11, B11 + B12, B21 + B22 (children 1, 3, 4,
// 6, 7) by complete mixed additions, normalised to canonical affine two
// points per lane at a time (one warp inversion per 64 points).  Parent and
// child arrays are quad-planar with np_count and nc_count ciphertexts.
__global__ void __launch_bounds__(128) strassen_csum_kernel(const uint4* __restrict__ B, int np, int lp,
                                                            long long nodes, uint4* __restrict__ T) {
    const int nh = np / 2, lh = lp / 2;
    const long long total = nodes * nh * lh;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < total;
    const long long tt = valid ? t : 0;
    const int j = (int)(tt % lh);
    const int k = (int)((tt / lh) % nh);
    const long long q = tt / ((long long)lh * nh);
    const size_t Np = (size_t)nodes * np * lp, Nc = (size_t)7 * nodes * nh * lh, cs = (size_t)nh * lh;
    const size_t i11 = ((size_t)q * np + k) * lp + j, i12 = i11 + lh;
    const size_t i21 = ((size_t)q * np + nh + k) * lp + j, i22 = i21 + lh;
    const size_t o = (size_t)7 * q * cs + (size_t)k * lh + j;    // child 1's element
    // Children 2 and 5 are copies.
#pragma unroll
    for (int c = 0; c < 2; c++) {
        aff x;
        load_aff(x, B + (size_t)c * 4 * Np, Np, i11);
        if (valid) store_aff(T + (size_t)c * 4 * Nc, Nc, o + 1 * cs, x);
        load_aff(x, B + (size_t)c * 4 * Np, Np, i22);
        if (valid) store_aff(T + (size_t)c * 4 * Nc, Nc, o + 4 * cs, x);
    }
    const size_t sx[5] = {i11, i12, i21, i11, i21};
    const size_t sy[5] = {i22, i22, i11, i12, i22};
    const bool neg[5] = {false, true, true, false, false};
    const int child[5] = {0, 2, 3, 5, 6};
#pragma unroll 1
    for (int u = 0; u < 5; u++) {
        jac R[2];
#pragma unroll
        for (int c = 0; c < 2; c++) {
            aff x, y;
            load_aff(x, B + (size_t)c * 4 * Np, Np, sx[u]);
            load_aff(y, B + (size_t)c * 4 * Np, Np, sy[u]);
            if (neg[u]) aff_negate(y);
            jac_from_aff(R[c], x);
            jac_madd(R[c], y);
        }
        aff out[2];
        warp_normalize_regs<2>(out, R);
        if (valid) {
#pragma unroll
            for (int c = 0; c < 2; c++) store_aff(T + (size_t)c * 4 * Nc, Nc, o + (size_t)child[u] * cs, out[c]);
        }
    }
}

// Leaf products of the deepest level: for each of the `leaves` nodes, the
// signed schoolbook product of its plaintext block (md x nd) and ciphertext
// block (nd x ld_): one warp per (leaf, row i, component c, 32 columns),
// each term |a| P by double-and-add, negated when a < 0, added by a
// complete Jacobian addition.  With no recursion (TOP: level 0) the
// plaintext is A itself, masked to w bits.
template <class TA, bool TOP>
__global__ void __launch_bounds__(128) strassen_leaf_kernel(const TA* __restrict__ S, int md, int nd, int ld_,
                                                            long long leaves, uint32_t amask,
                                                            const uint4* __restrict__ T,
                                                            uint4* __restrict__ M, uint32_t* status) {
    const unsigned lane = threadIdx.x & 31u;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int njb = (ld_ + 31) / 32;
    if (gw >= leaves * md * 2 * njb) return;
    const int jb = (int)(gw % njb);
    const int c = (int)((gw / njb) % 2);
    const int i = (int)((gw / (2 * njb)) % md);
    const long long q = gw / ((long long)2 * njb * md);
    const int j = jb * 32 + (int)lane;
    const int jj = j < ld_ ? j : ld_ - 1;
    const size_t NT = (size_t)leaves * nd * ld_, NM = (size_t)leaves * md * ld_;
    const uint4* Tc = T + (size_t)c * 4 * NT;
    const TA* a_row = S + ((size_t)q * md + i) * nd;
    jac acc, term;
    jac_set_inf(acc);
    aff P;
    for (int k = 0; k < nd; k++) {
        int a;
        if (TOP) {
            const uint32_t v = (uint32_t)a_row[k];
            if ((v & ~amask) && lane == 0 && c == 0 && jb == 0) atomicOr(status, DEV_ERR_A_RANGE);
            a = (int)(v & amask);
        } else {
            a = (int)a_row[k];
        }
        if (a == 0) continue;
        load_aff(P, Tc, NT, ((size_t)q * nd + k) * ld_ + jj);
        jac_mul_small(term, P, (uint32_t)(a < 0 ? -a : a));
        if (a < 0) {
            fe z;
            fe_zero(z);
            fe_sub(term.Y, z, term.Y);
        }
        jac_add(acc, term);
    }
    if (j < ld_) store_jac(M + (size_t)c * 6 * NM, NM, ((size_t)q * md + i) * ld_ + j, acc);
}

// One step up: every parent node's product from its seven children's,
// quadrant by quadrant (C11 = M1 + M4 - M5 + M7, C12 = M3 + M5,
// C21 = M2 + M4, C22 = M1 - M2 + M3 + M6) by complete Jacobian additions;
// one thread per (parent q, position (i, j) of a quadrant, component c).
__global__ void __launch_bounds__(128) strassen_combine_kernel(const uint4* __restrict__ M, int mc, int lc,
                                                               long long nodes, uint4* __restrict__ C) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nodes * mc * lc * 2) return;
    const int j = (int)(t % lc);
    const int i = (int)((t / lc) % mc);
    const int c = (int)((t / ((long long)lc * mc)) % 2);
    const long long q = t / ((long long)lc * mc * 2);
    const size_t NM = (size_t)7 * nodes * mc * lc, NC = (size_t)nodes * 4 * mc * lc, cs = (size_t)mc * lc;
    const uint4* Mc = M + (size_t)c * 6 * NM;
    uint4* Cc = C + (size_t)c * 6 * NC;
    const size_t m0 = (size_t)7 * q * cs + (size_t)i * lc + j;
    // Quadrant rows: children (1-based) and signs.
    const int terms[4][4] = {{1, 4, -5, 7}, {3, 5, 0, 0}, {2, 4, 0, 0}, {1, -2, 3, 6}};
    const int qi[4] = {0, 0, 1, 1}, qj[4] = {0, 1, 0, 1};
#pragma unroll 1
    for (int u = 0; u < 4; u++) {
        jac acc, x;
        jac_set_inf(acc);
        for (int v = 0; v < 4; v++) {
            const int r = terms[u][v];
            if (r == 0) continue;
            load_jac(x, Mc, NM, m0 + (size_t)((r < 0 ? -r : r) - 1) * cs);
            if (r < 0) {
                fe z;
                fe_zero(z);
                fe_sub(x.Y, z, x.Y);
            }
            jac_add(acc, x);
        }
        const size_t out = ((size_t)q * 2 * mc + (size_t)qi[u] * mc + i) * (2 * (size_t)lc) + (size_t)qj[u] * lc + j;
        store_jac(Cc, NC, out, acc);
    }
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace: a 256-byte header (status word), then per level t = 1..d the
// plaintext blocks (psum_bytes each, 7^t x m_t x n_t), the affine ciphertext blocks
// (7^t x n_t x l_t, 128 bytes each) and the Jacobian products
// (7^t x m_t x l_t, 192 bytes each), with m_t = m / 2^t and so on.
struct StrassenLayout {
    int d;
    long long nodes[STRASSEN_MAX_LEVELS + 1];
    int m[STRASSEN_MAX_LEVELS + 1], n[STRASSEN_MAX_LEVELS + 1], l[STRASSEN_MAX_LEVELS + 1];
    size_t offP[STRASSEN_MAX_LEVELS + 1], offB[STRASSEN_MAX_LEVELS + 1], offM[STRASSEN_MAX_LEVELS + 1];
    size_t bytes;
};

// Bytes of one plaintext block-sum entry: the sums of level t are below
// 2^(w + t) in magnitude, so int16 while w + levels <= 15, else int32.
inline int psum_bytes(int w, int levels) { return w + levels <= 15 ? 2 : 4; }

bool strassen_layout(StrassenLayout& L, int m, int n, int l, int w, int levels) {
    if (m < 1 || n < 1 || l < 1 || w < 1 || w > PCMM_MAX_W16 || levels < 0 || levels > STRASSEN_MAX_LEVELS)
        return false;
    const int pb = psum_bytes(w, levels);
    const int div = 1 << levels;
    if (m % div || n % div || l % div) return false;
    L.d = levels;
    size_t off = 256;
    long long nodes = 1;
    for (int t = 0; t <= levels; t++) {
        L.nodes[t] = nodes;
        L.m[t] = m >> t;
        L.n[t] = n >> t;
        L.l[t] = l >> t;
        if (t > 0) {
            L.offP[t] = off; off = a256(off + (size_t)nodes * L.m[t] * L.n[t] * pb);
            L.offB[t] = off; off = a256(off + (size_t)nodes * L.n[t] * L.l[t] * 128);
            L.offM[t] = off; off = a256(off + (size_t)nodes * L.m[t] * L.l[t] * 192);
        }
        nodes *= 7;
    }
    L.bytes = off;
    return true;
}

inline unsigned blocks_for(long long threads) { return (unsigned)((threads + 127) / 128); }

}  // namespace

extern "C" size_t pcmm_strassen_workspace_bytes(int m, int n, int l, int w, int levels) {
    StrassenLayout L;
    return strassen_layout(L, m, n, l, w, levels) ? L.bytes : 0;
}

namespace {

// The launches of one call: TA is A's element type, TS the block-sum type.
template <class TA, class TS>
pcmm_status strassen_run(const StrassenLayout& L, const TA* A, int w, const uint32_t* ctB, uint32_t* ctC,
                         uint8_t* base, cudaStream_t st) {
    uint32_t* status = (uint32_t*)base;
    const uint32_t amask = (uint32_t)((1ull << w) - 1u);
    if (cudaMemsetAsync(status, 0, 4, st) != cudaSuccess) return PCMM_ECUDA;
    // Down: block sums level by level.
    for (int t = 0; t < L.d; t++) {
        const long long pn = L.nodes[t];
        TS* S = (TS*)(base + L.offP[t + 1]);
        uint4* T = (uint4*)(base + L.offB[t + 1]);
        const uint4* B = t == 0 ? (const uint4*)ctB : (const uint4*)(base + L.offB[t]);
        ProfScope ps(KID_STRASSEN_SUM, st);
        const long long pthreads = pn * (L.m[t] / 2) * (L.n[t] / 2);
        if (t == 0)
            strassen_psum_kernel<TA, TS, true><<<blocks_for(pthreads), 128, 0, st>>>(A, L.m[0], L.n[0], pn, amask,
                                                                                   S, status);
        else
            strassen_psum_kernel<TS, TS, false><<<blocks_for(pthreads), 128, 0, st>>>(
                (const TS*)(base + L.offP[t]), L.m[t], L.n[t], pn, amask, S, status);
        PCMM_CUDA_CHECK_LAUNCH();
        const long long cthreads = pn * (L.n[t] / 2) * (L.l[t] / 2);
        strassen_csum_kernel<<<blocks_for(cthreads), 128, 0, st>>>(B, L.n[t], L.l[t], pn, T);
        PCMM_CUDA_CHECK_LAUNCH();
    }
    // Leaves.
    {
        const int d = L.d;
        const long long leaf_warps = L.nodes[d] * L.m[d] * 2 * ((L.l[d] + 31) / 32);
        uint4* M = d == 0 ? (uint4*)ctC : (uint4*)(base + L.offM[d]);
        ProfScope ps(KID_STRASSEN_LEAF, st);
        const unsigned blocks = (unsigned)((leaf_warps + 3) / 4);
        if (d == 0)
            strassen_leaf_kernel<TA, true><<<blocks, 128, 0, st>>>(A, L.m[0], L.n[0], L.l[0], 1, amask,
                                                                   (const uint4*)ctB, M, status);
        else
            strassen_leaf_kernel<TS, false><<<blocks, 128, 0, st>>>((const TS*)(base + L.offP[d]), L.m[d], L.n[d],
                                                                    L.l[d], L.nodes[d], amask,
                                                                    (const uint4*)(base + L.offB[d]), M, status);
        PCMM_CUDA_CHECK_LAUNCH();
    }
    // Up: each level's products from its children's.
    for (int t = L.d - 1; t >= 0; t--) {
        const uint4* M = (const uint4*)(base + L.offM[t + 1]);
        uint4* C = t == 0 ? (uint4*)ctC : (uint4*)(base + L.offM[t]);
        const int mc = L.m[t + 1], lc = L.l[t + 1];
        ProfScope ps(KID_STRASSEN_COMBINE, st);
        strassen_combine_kernel<<<blocks_for(L.nodes[t] * mc * lc * 2), 128, 0, st>>>(M, mc, lc, L.nodes[t], C);
        PCMM_CUDA_CHECK_LAUNCH();
    }
    return PCMM_OK;
}

template <class TA>
pcmm_status strassen_call(const TA* A, int m, int n, int w, const uint32_t* ctB, int l, uint32_t* ctC, int levels,
                          void* ws, size_t ws_bytes, pcmm_stream_t stream) {
    if (!A || !ctB || !ctC || !ws || ((uintptr_t)ws & 255u)) return PCMM_EINVAL;
    if (w > 8 * (int)sizeof(TA)) return PCMM_EINVAL;
    StrassenLayout L;
    if (!strassen_layout(L, m, n, l, w, levels)) return PCMM_EINVAL;
    if (ws_bytes < L.bytes) return PCMM_ENOMEM;
    // Every launch must fit the grid's x dimension (128-thread blocks).
    const long long max_blocks = 0x7fffffffLL;
    const long long leaf_warps = L.nodes[L.d] * L.m[L.d] * 2 * ((L.l[L.d] + 31) / 32);
    if ((leaf_warps + 3) / 4 > max_blocks) return PCMM_EUNSUPPORTED;
    for (int t = 0; t < L.d; t++) {
        const long long sums = L.nodes[t] * (L.m[t] / 2) * (L.n[t] / 2);
        const long long csums = L.nodes[t] * (L.n[t] / 2) * (L.l[t] / 2);
        const long long combine = L.nodes[t] * L.m[t + 1] * L.l[t + 1] * 2;
        if ((sums + 127) / 128 > max_blocks || (csums + 127) / 128 > max_blocks || (combine + 127) / 128 > max_blocks)
            return PCMM_EUNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (psum_bytes(w, levels) == 2) return strassen_run<TA, int16_t>(L, A, w, ctB, ctC, (uint8_t*)ws, st);
    return strassen_run<TA, int32_t>(L, A, w, ctB, ctC, (uint8_t*)ws, st);
}

}  // namespace

extern "C" pcmm_status pcmm_strassen(const uint8_t* A, int m, int n, int w, const uint32_t* ctB, int l,
                                     uint32_t* ctC, int levels, void* ws, size_t ws_bytes, pcmm_stream_t stream) {
    return strassen_call(A, m, n, w, ctB, l, ctC, levels, ws, ws_bytes, stream);
}

extern "C" pcmm_status pcmm_strassen16(const uint16_t* A, int m, int n, int w, const uint32_t* ctB, int l,
                                       uint32_t* ctC, int levels, void* ws, size_t ws_bytes, pcmm_stream_t stream) {
    return strassen_call(A, m, n, w, ctB, l, ctC, levels, ws, ws_bytes, stream);
}
