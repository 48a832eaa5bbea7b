// Device code of Cussen's compression-reconstruction PC-MM shared by the
// single-instance kernels (k_cussen.cu) and the persistent batched kernel
// (k_batched.cu): workspace layout, the plan of one strip, the table build of
// one warp item and the gather of one warp item.
#pragma once
#include <cuda_runtime.h>

#include <math.h>

#include "common.cuh"

namespace pcmm {
namespace cussen {

constexpr int NLEV = PCMM_N_ITER;   // compression iterations N

// Which field operations the gather's mixed addition and the table build's
// chain additions inline (build-time switches, see jacz_madd_t).  Measured
// on GB300 (w in {8, 4}, 1024 x 1024 x 256): gather 109.3 ms per step all out
// of line, 108.3 with the squarings inlined, 108.2 with a b - c d, 107.4-107.7
// with both (3), 112.5-127.8 when multiplications are inlined as well.
#ifndef PCMM_GATHER_INLINE
#define PCMM_GATHER_INLINE 3
#endif
#ifndef PCMM_TABLE_INLINE
#define PCMM_TABLE_INLINE 0
#endif
constexpr uint16_t NO_RANK = 0xFFFFu;
constexpr int PLAN_THREADS = 256;

struct Layout {
    int m, n, l, w, k;
    int nstrips, n1max, l2max, emax, lp, njb, ptr_stride;
    size_t off_rank, off_nent, off_codes, off_len, off_vN, off_ptr, off_rank1, plan_bytes;
    size_t item_u4, items_per_strip, table_points_per_strip, per_strip_bytes;
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Largest d with d (d + 1) / 2 <= 2^w - 1: the distinct positive differences
// of distinct values below 2^w sum to at most 2^w - 1, so every level after
// the first holds at most d entries.
inline int level2_bound(int w) {
    int lim = (1 << w) - 1, d = 0;
    while ((d + 1) * (d + 2) / 2 <= lim) d++;
    return d < 1 ? 1 : d;
}

// Workspace layout of one PC-MM (host and device agree on it).  Entries of A
// have up to PCMM_MAX_W16 bits; a strip code has w k <= PCMM_MAX_WK bits.
// Per column the plan holds the level lengths, the level-N values (uint16,
// l2max per column) and the tracking pointers of levels 1..N-1 (uint16:
// n1max for level 1, then l2max per further level).
inline bool make_layout(Layout& L, int m, int n, int l, int w, int k) {
    if (m < 1 || n < 1 || l < 1 || w < 1 || w > PCMM_MAX_W16 || k < 1 || w * k > PCMM_MAX_WK) return false;
    L.m = m; L.n = n; L.l = l; L.w = w; L.k = k;
    L.nstrips = (n + k - 1) / k;
    L.n1max = (1 << w) - 1 < m ? (1 << w) - 1 : m;
    L.l2max = level2_bound(w) < L.n1max ? level2_bound(w) : L.n1max;
    L.emax = (1 << (w * k)) - 1 < m ? (1 << (w * k)) - 1 : m;
    L.ptr_stride = L.n1max + (NLEV > 2 ? NLEV - 2 : 0) * L.l2max;
    L.njb = (l + 31) / 32;
    L.lp = L.njb * 32;
    size_t off = 256;  // status word and padding
    L.off_rank = off;  off = align256(off + (size_t)L.nstrips * m * 2);
    L.off_nent = off;  off = align256(off + (size_t)L.nstrips * 4);
    L.off_codes = off; off = align256(off + (size_t)L.nstrips * L.emax * 2);
    L.off_len = off;   off = align256(off + (size_t)n * NLEV * 2);
    L.off_vN = off;    off = align256(off + (size_t)n * L.l2max * 2);
    L.off_ptr = off;   off = align256(off + (size_t)n * L.ptr_stride * 2);
    L.off_rank1 = off; off = align256(off + (k > 1 ? (size_t)n * 256 : 0));
    L.plan_bytes = off;
    // Per warp item (lane-planar): Jacobian column table and level ping-pong;
    // affine level-2 entries, affine column tables and tuple partial sums
    // (k > 1); prefix products for the normalisations.
    const size_t jac_ents = (size_t)L.n1max + 2 * (size_t)L.l2max;
    const size_t aff_ents = (size_t)L.l2max + (k > 1 ? (size_t)k * L.n1max + (size_t)L.emax : 0);
    const size_t pref_ents = (size_t)(L.emax > L.n1max ? L.emax : L.n1max);
    L.item_u4 = jac_ents * 6 * 32 + aff_ents * 4 * 32 + pref_ents * 2 * 32;
    L.items_per_strip = 2 * (size_t)L.njb;
    L.table_points_per_strip = (size_t)L.emax * 2 * L.lp;
    L.per_strip_bytes = L.items_per_strip * L.item_u4 * 16 + align256(L.table_points_per_strip * 64);
    return true;
}

struct PlanPtrs {
    uint32_t* status;
    uint16_t* rank;
    int32_t* nent;
    uint16_t* codes;
    uint16_t* col_len;
    uint16_t* col_vN;      // [col][l2max]
    uint16_t* col_ptr;     // [col][ptr_stride]
    uint8_t* col_rank1;    // [col][256] (k > 1, so w <= 8)
    int n1max, l2max, ptr_stride, emax;
};

inline PlanPtrs plan_ptrs(const Layout& L, void* ws) {
    uint8_t* b = (uint8_t*)ws;
    PlanPtrs P;
    P.status = (uint32_t*)b;
    P.rank = (uint16_t*)(b + L.off_rank);
    P.nent = (int32_t*)(b + L.off_nent);
    P.codes = (uint16_t*)(b + L.off_codes);
    P.col_len = (uint16_t*)(b + L.off_len);
    P.col_vN = (uint16_t*)(b + L.off_vN);
    P.col_ptr = (uint16_t*)(b + L.off_ptr);
    P.col_rank1 = b + L.off_rank1;
    P.n1max = L.n1max;
    P.l2max = L.l2max;
    P.ptr_stride = L.ptr_stride;
    P.emax = L.emax;
    return P;
}

// Tracking pointers of level lev (1 .. NLEV-1) of column col: entry e of
// level lev sits at position ptr[e] of level lev + 1.
__device__ __forceinline__ uint16_t* col_level_ptr(const PlanPtrs& P, int col, int lev) {
    return P.col_ptr + (size_t)col * P.ptr_stride + (lev == 1 ? 0 : P.n1max + (size_t)(lev - 2) * P.l2max);
}

__device__ __forceinline__ int warp_excl_scan(int v, int& total) {
    const unsigned lane = threadIdx.x & 31u;
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, incl, d);
        if ((int)lane >= d) incl += o;
    }
    total = __shfl_sync(0xffffffffu, incl, 31);
    return incl - v;
}

// Sorted list of the values marked in a 256-bit presence map; also a
// value -> position map.  Each lane owns 8 consecutive values.
__device__ __forceinline__ int extract_sorted(const uint32_t* bm, uint16_t* out, uint8_t* pos_of) {
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t bits8 = (bm[lane >> 2] >> ((lane & 3u) * 8u)) & 0xffu;
    int total;
    int pos = warp_excl_scan(__popc(bits8), total);
    for (int b = 0; b < 8; b++) {
        if ((bits8 >> b) & 1u) {
            const int v = (int)lane * 8 + b;
            out[pos] = (uint16_t)v;
            pos_of[v] = (uint8_t)pos;
            pos++;
        }
    }
    __syncwarp();
    return total;
}

// ---- block-level helpers of the plan (blockDim.x == PLAN_THREADS) ----

// Exclusive prefix sum of one value per thread over the block; every thread
// receives the total.  All threads must call.
__device__ __forceinline__ int block_excl_scan(int v, int& total) {
    __shared__ int wsum[PLAN_THREADS / 32];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    int wt;
    const int x = warp_excl_scan(v, wt);
    __syncthreads();
    if (lane == 0) wsum[warp] = wt;
    __syncthreads();
    int base = 0, tot = 0;
    for (int q = 0; q < PLAN_THREADS / 32; q++) {
        const int t = wsum[q];
        if (q < (int)warp) base += t;
        tot += t;
    }
    total = tot;
    return base + x;
}

// Exclusive prefix maximum (identity -1) of one value per thread.
__device__ __forceinline__ int block_excl_max(int v) {
    __shared__ int wmax[PLAN_THREADS / 32];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, d);
        if ((int)lane >= d) incl = o > incl ? o : incl;
    }
    int ex = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) ex = -1;
    __syncthreads();
    if (lane == 31) wmax[warp] = incl;
    __syncthreads();
    for (int q = 0; q < (int)warp; q++) ex = wmax[q] > ex ? wmax[q] : ex;
    return ex;
}

// Words [w0, w0 + wpt) of an nw-word presence map belong to this thread.
__device__ __forceinline__ int map_words_per_thread(int nw) { return (nw + PLAN_THREADS - 1) / PLAN_THREADS; }

// pf[x] = number of set bits in words 0..x-1 of bm; returns the total.
__device__ __forceinline__ int map_prefix(const uint32_t* bm, uint32_t* pf, int nw) {
    const int wpt = map_words_per_thread(nw);
    const int w0 = (int)threadIdx.x * wpt;
    int cnt = 0;
    for (int q = 0; q < wpt; q++)
        if (w0 + q < nw) cnt += __popc(bm[w0 + q]);
    int total;
    int base = block_excl_scan(cnt, total);
    for (int q = 0; q < wpt; q++)
        if (w0 + q < nw) {
            pf[w0 + q] = (uint32_t)base;
            base += __popc(bm[w0 + q]);
        }
    __syncthreads();
    return total;
}

// Position of the present value v in the sorted list of present values.
__device__ __forceinline__ int map_rank(const uint32_t* bm, const uint32_t* pf, uint32_t v) {
    return (int)(pf[v >> 5] + __popc(bm[v >> 5] & ((1u << (v & 31u)) - 1u)));
}

__device__ __forceinline__ void map_clear(uint32_t* bm, int nw) {
    for (int x = threadIdx.x; x < nw; x += PLAN_THREADS) bm[x] = 0u;
}

// Levels 2..N of one column whose values have up to 16 bits (w > 8, hence
// k = 1), computed by the whole block.  Level 1 (the sorted distinct
// non-zero values) is given as the presence map bm1 of nw words with its
// prefix counts pf1.  Level q + 1 is the sorted distinct set of the
// differences of consecutive level-q values (the first minus zero); the
// tracking pointer of a level-q entry is the position of its difference in
// level q + 1.  bm/pf: nw-word work maps; lvA/lvB: lists of l2max entries.
__device__ __forceinline__ void plan_column_wide(const uint32_t* bm1, const uint32_t* pf1, int nw, int len1,
                                                 int col, const PlanPtrs& P, uint32_t* bm, uint32_t* pf,
                                                 uint16_t* lvA, uint16_t* lvB) {
    const int wpt = map_words_per_thread(nw);
    const int w0 = (int)threadIdx.x * wpt;
    if (threadIdx.x == 0) P.col_len[(size_t)col * NLEV] = (uint16_t)len1;
    // Level 1 -> 2.  The predecessor of the first value in this thread's
    // words is the largest value in the words before them.
    int last = -1;
    for (int q = 0; q < wpt; q++)
        if (w0 + q < nw && bm1[w0 + q]) last = (w0 + q) * 32 + 31 - __clz(bm1[w0 + q]);
    const int prev0 = block_excl_max(last);
    map_clear(bm, nw);
    __syncthreads();
    for (int pass = 0; pass < 2; pass++) {
        int prev = prev0 < 0 ? 0 : prev0;
        uint16_t* ptr1 = col_level_ptr(P, col, 1);
        for (int q = 0; q < wpt; q++) {
            if (w0 + q >= nw) break;
            uint32_t x = bm1[w0 + q];
            while (x) {
                const uint32_t v = (uint32_t)(w0 + q) * 32u + (uint32_t)(__ffs(x) - 1);
                const uint32_t d = v - (uint32_t)prev;
                if (pass == 0) atomicOr(&bm[d >> 5], 1u << (d & 31u));
                else ptr1[map_rank(bm1, pf1, v)] = (uint16_t)map_rank(bm, pf, d);
                prev = (int)v;
                x &= x - 1u;
            }
        }
        __syncthreads();
        if (pass == 0) map_prefix(bm, pf, nw);
    }
    uint16_t* cur = lvA;
    uint16_t* nxt = lvB;
    int len = 0;
    for (int lev = 1; lev < NLEV; lev++) {
        if (lev > 1) {
            // Differences of the level-lev list into the work map.
            map_clear(bm, nw);
            __syncthreads();
            for (int e = threadIdx.x; e < len; e += PLAN_THREADS) {
                const uint32_t d = (uint32_t)cur[e] - (e ? (uint32_t)cur[e - 1] : 0u);
                atomicOr(&bm[d >> 5], 1u << (d & 31u));
            }
            __syncthreads();
            map_prefix(bm, pf, nw);
            uint16_t* ptr = col_level_ptr(P, col, lev);
            for (int e = threadIdx.x; e < len; e += PLAN_THREADS) {
                const uint32_t d = (uint32_t)cur[e] - (e ? (uint32_t)cur[e - 1] : 0u);
                ptr[e] = (uint16_t)map_rank(bm, pf, d);
            }
        }
        // Level lev + 1: the sorted present values of the work map.
        int nlen;
        {
            int cnt = 0;
            for (int q = 0; q < wpt; q++)
                if (w0 + q < nw) cnt += __popc(bm[w0 + q]);
            block_excl_scan(cnt, nlen);
        }
        for (int q = 0; q < wpt; q++) {
            if (w0 + q >= nw) break;
            uint32_t x = bm[w0 + q];
            while (x) {
                const uint32_t d = (uint32_t)(w0 + q) * 32u + (uint32_t)(__ffs(x) - 1);
                const int r = map_rank(bm, pf, d);
                if (r < P.l2max) nxt[r] = (uint16_t)d;
                x &= x - 1u;
            }
        }
        if (threadIdx.x == 0) P.col_len[(size_t)col * NLEV + lev] = (uint16_t)nlen;
        __syncthreads();
        uint16_t* tmp = cur; cur = nxt; nxt = tmp;
        len = nlen < P.l2max ? nlen : P.l2max;
    }
    for (int e = threadIdx.x; e < len; e += PLAN_THREADS) P.col_vN[(size_t)col * P.l2max + e] = cur[e];
    __syncthreads();
}

// Block-level plan of strip s (all PLAN_THREADS threads of the block call):
// the presence map of the strip's codes (a code is the k-tuple of a row's
// entries, w bits each), each row's rank among the distinct non-zero codes,
// the list of distinct codes (k > 1) and the compression levels of every
// column of the strip.  TA is the element type of A (uint8 or uint16).
template <class TA>
__device__ __forceinline__ void plan_strip(const TA* __restrict__ A, int m, int n, int w, int k,
                                           const PlanPtrs& P, int s) {
    constexpr int MAP_WORDS = 1 << (PCMM_MAX_WK - 5);
    __shared__ uint32_t spres[MAP_WORDS];
    __shared__ uint32_t spref[MAP_WORDS];
    __shared__ uint32_t work[2 * MAP_WORDS];
    __shared__ uint16_t lv[2][512];
    const int c0 = s * k;
    const int kw = (c0 + k <= n) ? k : n - c0;
    const uint32_t amask = (1u << w) - 1u;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const int emax = P.emax;

    // ---- strip codes, distinct codes and per-row ranks ----
    const int cbits = w * k;
    const int nwc = cbits > 5 ? 1 << (cbits - 5) : 1;
    map_clear(spres, nwc);
    __syncthreads();
    bool bad = false;
    for (int i = threadIdx.x; i < m; i += PLAN_THREADS) {
        uint32_t code = 0;
        for (int t = 0; t < kw; t++) {
            const uint32_t v = (uint32_t)A[(size_t)i * n + c0 + t];
            bad |= v > amask;
            code |= (v & amask) << (w * t);
        }
        if (code) atomicOr(&spres[code >> 5], 1u << (code & 31u));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(P.status, DEV_ERR_A_RANGE);
    const int total = map_prefix(spres, spref, nwc);
    if (threadIdx.x == 0) P.nent[s] = total;
    for (int i = threadIdx.x; i < m; i += PLAN_THREADS) {
        uint32_t code = 0;
        for (int t = 0; t < kw; t++) code |= ((uint32_t)A[(size_t)i * n + c0 + t] & amask) << (w * t);
        P.rank[(size_t)s * m + i] = code ? (uint16_t)map_rank(spres, spref, code) : NO_RANK;
    }
    if (k > 1) {
        for (int wd = threadIdx.x; wd < nwc; wd += PLAN_THREADS) {
            uint32_t bits = spres[wd];
            uint32_t r = spref[wd];
            while (bits) {
                const int b = __ffs(bits) - 1;
                if ((int)r < emax) P.codes[(size_t)s * emax + r] = (uint16_t)(wd * 32 + b);
                r++;
                bits &= bits - 1u;
            }
        }
    }

    if (w > 8) {
        // ---- wide values: k = 1, the strip map is the column's level 1 ----
        plan_column_wide(spres, spref, 1 << (w - 5), total, c0, P, work, work + MAP_WORDS, lv[0], lv[1]);
        return;
    }

    // ---- narrow values: per-column levels, one warp per column ----
    uint32_t* wbm = work + warp * 8;                                                   // 8 words
    uint16_t* wlev = (uint16_t*)(work + 64) + (size_t)warp * 512;                      // 2 x 256
    uint8_t* pos = (uint8_t*)(work + 64 + 256 * (PLAN_THREADS / 32)) + (size_t)warp * 256;
    for (int t = (int)warp; t < kw; t += PLAN_THREADS / 32) {
        const int col = c0 + t;
        uint32_t* bm = wbm;
        if (lane < 8) bm[lane] = 0u;
        __syncwarp();
        for (int i = (int)lane; i < m; i += 32) {
            const uint32_t v = (uint32_t)A[(size_t)i * n + col] & amask;
            if (v) atomicOr(&bm[v >> 5], 1u << (v & 31u));
        }
        __syncwarp();
        uint16_t* cur = wlev;
        uint16_t* nxt = wlev + 256;
        int len = extract_sorted(bm, cur, pos);
        if (k > 1) {
            // value -> level-1 position, for the k-tuple assembly
            for (int v = (int)lane; v < 256; v += 32) {
                const bool present = v > 0 && ((bm[v >> 5] >> (v & 31)) & 1u);
                P.col_rank1[(size_t)col * 256 + v] = present ? pos[v] : (uint8_t)0xff;
            }
        }
        if (lane == 0) P.col_len[(size_t)col * NLEV] = (uint16_t)len;
        __syncwarp();
        for (int lev = 1; lev < NLEV; lev++) {
            // Differences of consecutive sorted values; level lev + 1 is their
            // sorted distinct set.
            if (lane < 8) bm[lane] = 0u;
            __syncwarp();
            for (int e = (int)lane; e < len; e += 32) {
                const int d = (int)cur[e] - (e ? (int)cur[e - 1] : 0);
                atomicOr(&bm[d >> 5], 1u << (d & 31));
            }
            __syncwarp();
            const int nlen = extract_sorted(bm, nxt, pos);
            uint16_t* ptr = col_level_ptr(P, col, lev);
            for (int e = (int)lane; e < len; e += 32) {
                const int d = (int)cur[e] - (e ? (int)cur[e - 1] : 0);
                ptr[e] = pos[d];
            }
            if (lane == 0) P.col_len[(size_t)col * NLEV + lev] = (uint16_t)nlen;
            __syncwarp();
            uint16_t* tmp = cur; cur = nxt; nxt = tmp;
            len = nlen < P.l2max ? nlen : P.l2max;
        }
        for (int e = (int)lane; e < len; e += 32) P.col_vN[(size_t)col * P.l2max + e] = cur[e];
        __syncwarp();
    }
}

struct TableArgs {
    const uint4* ctB;      // affine ciphertext matrix n x l
    int m, n, l, w, k, lp, njb, n1max, l2max, emax;
    int s0, nstrips_chunk;
    uint4* scratch;        // lane-planar per-item scratch
    size_t item_u4;
    uint4* table;          // affine, quad-planar, table_points points
    size_t table_points;
    bool bshare;           // the 4 warps of each block share one strip's plan: share inversions
};

__device__ __forceinline__ void lp_store_aff(uint4* base, int e, unsigned lane, const aff& Q) {
    uint4* b = base + (size_t)e * 4 * 32 + lane;
    b[0] = fe_lo(Q.x);
    b[32] = fe_hi(Q.x);
    b[64] = fe_lo(Q.y);
    b[96] = fe_hi(Q.y);
}

__device__ __forceinline__ void lp_load_aff(aff& Q, const uint4* base, int e, unsigned lane) {
    const uint4* b = base + (size_t)e * 4 * 32 + lane;
    fe_from_quads(Q.x, b[0], b[32]);
    fe_from_quads(Q.y, b[64], b[96]);
}


// One forward step of the simultaneous inversion, for loops that produce
// lane-planar Jacobian entries: acc *= Z_e (a zero Z, i.e. infinity, counts
// as 1), prefix product stored as entry e of pref; ones tracks whether every
// Z so far is 1.
__device__ __forceinline__ void lp_pref_step(fe& acc, bool& ones, const fe& Z, uint4* pref, int e,
                                             unsigned lane) {
    fe z = Z;
    ones &= fe_is_one(z);
    if (fe_is_zero(z)) fe_one(z);
    acc = fmul(acc, z);
    lp_store_fe(pref, e, lane, acc);
}

// Backward half of the normalisation of E lane-planar Jacobian entries to
// canonical affine (infinity -> (0, 0)), each handed to store(e, point):
// pref holds the per-lane prefix products of the Z's and acc their total
// (lp_pref_step).  One warp-wide inversion; when every Z in the warp is 1 the
// entries are copied without any.  The loads of entry e - 2 are prefetched
// into L2 while entry e is converted (lanes 0-23: the 24 lines of the
// Jacobian entry, lanes 24-31: the 8 lines of its prefix product).  All 32
// lanes call with the same E.
template <class Store>
__device__ __forceinline__ void lp_normalize_back(const uint4* src, int E, const uint4* pref, unsigned lane,
                                                  fe acc, bool ones, Store store, bool shared) {
    if (E <= 0) return;
    if (group_all(ones, shared)) {
        for (int e = 0; e < E; e++) {
            jac Pe;
            lp_load_jac(Pe, src, e, lane);
            aff out;
            fe_canon(out.x, Pe.X);
            fe_canon(out.y, Pe.Y);
            store(e, out);
        }
        return;
    }
    fe inv;
    group_inverse(inv, acc, shared);
    for (int e = E - 1; e >= 0; e--) {
        if (e >= 2) {
            const char* line = lane < 24u ? (const char*)(src + (size_t)(e - 2) * 192) + lane * 128u
                                          : (e >= 3 ? (const char*)(pref + (size_t)(e - 3) * 64) + (lane - 24u) * 128u
                                                    : nullptr);
            if (line) asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
        }
        fe zinv;
        if (e > 0) {
            fe pr;
            lp_load_fe(pr, pref, e - 1, lane);
            zinv = fmul(inv, pr);
        } else {
            zinv = inv;
        }
        jac Pe;
        lp_load_jac(Pe, src, e, lane);
        fe z = Pe.Z;
        const bool is_inf = fe_is_zero(z);
        if (is_inf) fe_one(z);
        inv = fmul(inv, z);
        aff out;
        if (is_inf) {
            fe_zero(out.x);
            fe_zero(out.y);
        } else {
            jac_to_aff_with_zinv(out, Pe, zinv);
        }
        store(e, out);
    }
}

// Normalises E lane-planar Jacobian entries already in scratch (both passes).
template <class Store>
__device__ __forceinline__ void lp_normalize(const uint4* src, int E, uint4* pref, unsigned lane,
                                             Store store, bool shared) {
    if (E <= 0) return;
    bool ones = true;
    fe acc;
    fe_one(acc);
    for (int e = 0; e < E; e++) {
        fe z;
        lp_load_z(z, src, e, lane);
        lp_pref_step(acc, ones, z, pref, e, lane);
    }
    lp_normalize_back(src, E, pref, lane, acc, ones, store, shared);
}

// Normalises the E entries of a chain kept as (X, Y, ZZ, ZZZ)
// (jacz_madd_ratio_t): entry e holds X and Y in quads 0-3 of its 6-quad
// lane-planar slot in src and its ZZZ factor rr3_e in quads 4-5, and its ZZ
// factor rr2_e is entry e of rat, so ZZ_e = rr2_0 ... rr2_e (likewise ZZZ);
// zz, zzz are those of the last entry.  One inversion of zz zzz gives both
// ZZ^-1 and ZZZ^-1 of the last entry; going backwards each step multiplies
// them by the entry's factors: 4M per entry in all.  ones: every factor of
// this lane is 1.  With `shared` all threads of the block must call.
template <class Store>
__device__ __forceinline__ void lp_normalize_zz(const uint4* src, int E, const uint4* rat, unsigned lane,
                                                const fe& zz, const fe& zzz, bool ones, Store store,
                                                bool shared) {
    if (E <= 0) return;
    if (group_all(ones, shared)) {
        for (int e = 0; e < E; e++) {
            const uint4* b = src + (size_t)e * 6 * 32 + lane;
            aff out;
            fe_from_quads(out.x, b[0], b[32]);
            fe_from_quads(out.y, b[64], b[96]);
            fe_canon(out.x, out.x);
            fe_canon(out.y, out.y);
            store(e, out);
        }
        return;
    }
    fe inv;
    group_inverse(inv, fmul(zz, zzz), shared);
    fe zzinv = fmul(inv, zzz);
    fe zzzinv = fmul(inv, zz);
    for (int e = E - 1; e >= 0; e--) {
        if (e >= 2) {
            // lanes 0-23: the 24 lines of slot e - 2; 24-31: its ZZ factor.
            const char* line = lane < 24u ? (const char*)(src + (size_t)(e - 2) * 192) + lane * 128u
                                          : (const char*)(rat + (size_t)(e - 2) * 64) + (lane - 24u) * 128u;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(line));
        }
        const uint4* b = src + (size_t)e * 6 * 32 + lane;
        fe X, Y;
        fe_from_quads(X, b[0], b[32]);
        fe_from_quads(Y, b[64], b[96]);
        aff out;
        out.x = fmul(X, zzinv);
        out.y = fmul(Y, zzzinv);
        fe_canon(out.x, out.x);
        fe_canon(out.y, out.y);
        store(e, out);
        if (e > 0) {
            fe r2, r3;
            lp_load_fe(r2, rat, e, lane);
            fe_from_quads(r3, b[128], b[160]);
            zzinv = fmul(zzinv, r2);
            zzzinv = fmul(zzzinv, r3);
        }
    }
}

// The chain P_e = P_{e-1} + A[ptr[e]] (e < len, P_{-1} at infinity) over
// affine addends A (lane-planar, 4 quads per entry), in (X, Y, ZZ, ZZZ):
// entry e's X, Y and ZZZ factor go to slot e of `slots` (6 quads), its ZZ
// factor to entry e of rat, as lp_normalize_zz reads them.  acc ends as the
// last entry; ones and ok as for jacz_madd_ratio_t.
static __device__ __noinline__ void lp_affine_chain(const uint4* A, const uint16_t* ptr, int len, uint4* slots,
                                                    uint4* rat, unsigned lane, jacz& acc, bool& ones, bool& ok) {
    aff D;
    jacz_set_inf(acc);
    ones = true;
    ok = true;
    for (int e = 0; e < len; e++) {
        lp_load_aff(D, A, ptr[e], lane);
        fe r2, r3;
        jacz_madd_ratio_t<PCMM_TABLE_INLINE>(acc, D, r2, r3, ok, e == 0);
        uint4* b = slots + (size_t)e * 6 * 32 + lane;
        b[0] = fe_lo(acc.X);
        b[32] = fe_hi(acc.X);
        b[64] = fe_lo(acc.Y);
        b[96] = fe_hi(acc.Y);
        b[128] = fe_lo(r3);
        b[160] = fe_hi(r3);
        lp_store_fe(rat, e, lane, r2);
        ones &= fe_is_one(r2) && fe_is_one(r3);
    }
}

// One warp per (strip, component c, 32 output columns); all lanes follow the
// same plan, so the control flow is warp-uniform.
// Table of one warp item (strip, component, 32 output columns) of a chunk;
// `scratch` is this warp's private scratch (a.item_u4 uint4).
__device__ __forceinline__ void table_item(const TableArgs& a, const PlanPtrs& P, long long item,
                                           uint4* scratch) {
    static_assert(NLEV >= 2, "the table build assumes at least two compression levels");
    const unsigned lane = threadIdx.x & 31u;
    const int s_local = (int)(item / (2 * a.njb));
    const int rem = (int)(item % (2 * a.njb));
    const int c = rem / a.njb, jb = rem % a.njb;
    const int s = a.s0 + s_local;
    const int c0 = s * a.k;
    const int kw = (c0 + a.k <= a.n) ? a.k : a.n - c0;
    const int j = jb * 32 + (int)lane;
    const int jj = j < a.l ? j : a.l - 1;
    const size_t nl = (size_t)a.n * a.l;
    const uint4* Bc = a.ctB + (size_t)c * 4 * nl;
    const uint32_t amask = (1u << a.w) - 1u;

    // Scratch regions of this warp item (see make_layout).
    uint4* coltab = scratch;                                              // n1max Jacobian
    uint4* levA = coltab + (size_t)a.n1max * 192;                         // l2max Jacobian
    uint4* levB = levA + (size_t)a.l2max * 192;                           // l2max Jacobian
    uint4* l2aff = levB + (size_t)a.l2max * 192;                          // l2max affine
    uint4* colaff = l2aff + (size_t)a.l2max * 128;                        // k * n1max affine (k > 1)
    uint4* part = colaff + (a.k > 1 ? (size_t)a.k * a.n1max * 128 : 0);   // emax affine (k > 1)
    uint4* pref = part + (a.k > 1 ? (size_t)a.emax * 128 : 0);            // max(emax, n1max) field elements

    const int E = P.nent[s];
    const size_t tbase = (size_t)s_local * a.emax;
    auto store_table = [&](int e, const aff& q) {
        store_aff(a.table, a.table_points, ((tbase + e) * 2 + c) * a.lp + j, q);
    };
    bool bad = false, dbad = false;

    for (int t = 0; t < kw; t++) {
        const int col = c0 + t;
        aff Pb;
        load_aff(Pb, Bc, nl, (size_t)col * a.l + jj);
        int lens[NLEV];
#pragma unroll
        for (int q = 0; q < NLEV; q++) lens[q] = P.col_len[(size_t)col * NLEV + q];
        bad |= lens[0] > a.n1max;
#pragma unroll
        for (int q = 1; q < NLEV; q++) bad |= lens[q] > a.l2max;
#ifdef PCMM_DEBUG_BOUNDS
        // Each tracking pointer of level lev (lens[lev-1] of them) names an
        // entry of level lev + 1 (lens[lev] entries); for k = 1 the strip
        // table is the column's level 1.
        for (int lev = 1; lev < NLEV && !bad; lev++) {
            const uint16_t* pl = col_level_ptr(P, col, lev);
            for (int e = 0; e < lens[lev - 1]; e++) dbad |= pl[e] >= lens[lev];
        }
        if (a.k == 1) dbad |= E != lens[0];
        bad |= dbad;
#endif
        if (bad) break;
        // Level N: multiples of the compressed values (double-and-add).
        uint4* src = levA;
        for (int e = 0; e < lens[NLEV - 1]; e++) {
            jac T;
            jac_mul_small(T, Pb, P.col_vN[(size_t)col * P.l2max + e]);
            lp_store_jac(src, e, lane, T);
        }
        uint4* alt = levB;
        // Levels N-1..2: un-sort by the tracking pointers, then prefix sums of
        // Jacobian points; level 2 also takes the forward pass of its
        // normalisation.  A long level 2 (wide values: hundreds of entries) is
        // instead built like level 1, as a chain of mixed additions over its
        // level 3 normalised to affine (plan data, so uniform over the strip).
        const bool l2chain = NLEV > 2 && lens[1] >= 32;
        auto store_l2 = [&](int e, const aff& q) { lp_store_aff(l2aff, e, lane, q); };
        fe pacc;
        bool pones = true;
        fe_one(pacc);
        auto jacobian_level = [&](int lev) {
            const uint16_t* ptr = col_level_ptr(P, col, lev);
            jac acc, D;
            jac_set_inf(acc);
            for (int e = 0; e < lens[lev - 1]; e++) {
                lp_load_jac(D, src, ptr[e], lane);
                jac_add(acc, D);
                lp_store_jac(alt, e, lane, acc);
                if (lev == 2) lp_pref_step(pacc, pones, acc.Z, pref, e, lane);
            }
        };
        for (int lev = NLEV - 1; lev >= (l2chain ? 3 : 2); lev--) {
            jacobian_level(lev);
            uint4* tmp = src; src = alt; alt = tmp;
        }
        if (!l2chain) {
            // Level 2 (multiples of the level-1 differences) to affine, so that
            // the level-1 prefix sums are mixed additions.
            if (NLEV > 2) lp_normalize_back(src, lens[1], pref, lane, pacc, pones, store_l2, a.bshare);
            else lp_normalize(src, lens[1], pref, lane, store_l2, a.bshare);
        } else {
            // Level 3 (Jacobian, in src) to affine in l2aff, then level 2 as a
            // chain over it into alt; l2aff then receives level 2.
            lp_normalize(src, lens[2], pref, lane, store_l2, a.bshare);
            jacz acc2;
            bool ones2, ok2;
            lp_affine_chain(l2aff, col_level_ptr(P, col, 2), lens[1], alt, pref, lane, acc2, ones2, ok2);
            if (group_all(ok2, a.bshare)) {
                lp_normalize_zz(alt, lens[1], pref, lane, acc2.ZZ, acc2.ZZZ, ones2, store_l2, a.bshare);
            } else {
                jacobian_level(2);
                lp_normalize_back(alt, lens[1], pref, lane, pacc, pones, store_l2, a.bshare);
            }
        }
        // Level 1: the multiples of the column's sorted distinct values,
        // with the forward pass of their normalisation.
        // The chain runs in (X, Y, ZZ, ZZZ) coordinates; each entry keeps X,
        // Y and the factors its ZZ and ZZZ were multiplied by, for the
        // normalisation.  A chain that meets infinity (an input at infinity)
        // is recomputed in Jacobian coordinates and normalised the general way.
        const uint16_t* ptr1 = col_level_ptr(P, col, 1);
        jacz acc;
        bool cones, cok;
        lp_affine_chain(l2aff, ptr1, lens[0], coltab, pref, lane, acc, cones, cok);
        const bool chain_ok = group_all(cok, a.bshare);
        if (!chain_ok) {
            jac accj;
            aff D;
            jac_set_inf(accj);
            for (int e = 0; e < lens[0]; e++) {
                lp_load_aff(D, l2aff, ptr1[e], lane);
                jac_madd(accj, D);
                lp_store_jac(coltab, e, lane, accj);
            }
        }
        uint4* ca = colaff + (size_t)t * a.n1max * 128;
        auto store_col = [&](int e, const aff& q) { lp_store_aff(ca, e, lane, q); };
        if (a.k == 1) {
            // The column table is the strip table (E = lens[0] entries).
            if (chain_ok) lp_normalize_zz(coltab, E, pref, lane, acc.ZZ, acc.ZZZ, cones, store_table, a.bshare);
            else lp_normalize(coltab, E, pref, lane, store_table, a.bshare);
            return;
        }
        if (chain_ok) lp_normalize_zz(coltab, lens[0], pref, lane, acc.ZZ, acc.ZZZ, cones, store_col, a.bshare);
        else lp_normalize(coltab, lens[0], pref, lane, store_col, a.bshare);
    }
    if (bad) {
        if (lane == 0) atomicOr(P.status, dbad ? DEV_ERR_BOUNDS : DEV_ERR_PLAN);
        return;
    }
#ifdef PCMM_DEBUG_BOUNDS
    // Every component of every tuple names an entry of its column table.
    for (int e = 0; e < E && !dbad; e++) {
        const uint32_t code = P.codes[(size_t)s * a.emax + e];
        for (int t = 0; t < kw; t++) {
            const uint32_t x = (code >> (a.w * t)) & amask;
            if (x) dbad |= P.col_rank1[(size_t)(c0 + t) * 256 + x] >= P.col_len[(size_t)(c0 + t) * NLEV];
        }
    }
    if (E > a.emax || dbad) {
        if (lane == 0) atomicOr(P.status, DEV_ERR_BOUNDS);
        return;
    }
#endif
    // k > 1: one entry per distinct k-tuple, the sum of its columns' (affine)
    // entries, computed in affine coordinates one addition round at a time:
    // round r adds the (r+1)-th non-zero component of every tuple that has
    // one.  The additions of a round are independent, so their slopes share
    // one simultaneous inversion (per-lane prefix products of the x
    // differences, then one warp-wide inversion): about 5M + 1S per entry
    // instead of a mixed addition and a normalisation.  Pairs the affine
    // formula cannot take (infinity, equal or opposite points) use the
    // complete Jacobian addition and their own inversion on a rare branch.
    auto comp = [&](uint32_t code, int nth, uint32_t& v) -> int {
        int cnt = 0;
        for (int t = 0; t < kw; t++) {
            const uint32_t x = (code >> (a.w * t)) & amask;
            if (x) {
                if (cnt == nth) { v = x; return t; }
                cnt++;
            }
        }
        return -1;
    };
    auto col_entry = [&](aff& Q, int t, uint32_t v) {
        const int r1 = P.col_rank1[(size_t)(c0 + t) * 256 + v];
        lp_load_aff(Q, colaff + (size_t)t * a.n1max * 128, r1, lane);
    };
    int maxc = 0;
    for (int e = 0; e < E; e++) {
        const uint32_t code = P.codes[(size_t)s * a.emax + e];
        int cnt = 0;
        for (int t = 0; t < kw; t++) cnt += ((code >> (a.w * t)) & amask) != 0u;
        maxc = cnt > maxc ? cnt : maxc;
    }
    for (int r = 1; r < maxc; r++) {
        fe acc;
        fe_one(acc);
        for (int e = 0; e < E; e++) {
            const uint32_t code = P.codes[(size_t)s * a.emax + e];
            uint32_t vq, v0;
            const int tq = comp(code, r, vq);
            fe dx;
            fe_one(dx);
            if (tq >= 0) {
                aff Pp, Qq;
                if (r == 1) col_entry(Pp, comp(code, 0, v0), v0);
                else lp_load_aff(Pp, part, e, lane);
                col_entry(Qq, tq, vq);
                if (!aff_is_inf(Pp) && !aff_is_inf(Qq)) {
                    fe_sub(dx, Qq.x, Pp.x);
                    if (fe_is_zero(dx)) fe_one(dx);
                }
            }
            acc = fmul(acc, dx);
            lp_store_fe(pref, e, lane, acc);
        }
        fe inv;
        group_inverse(inv, acc, a.bshare);
        for (int e = E - 1; e >= 0; e--) {
            const uint32_t code = P.codes[(size_t)s * a.emax + e];
            uint32_t vq, v0;
            const int tq = comp(code, r, vq);
            if (tq < 0) continue;          // its factor was 1
            aff Pp, Qq, R;
            if (r == 1) col_entry(Pp, comp(code, 0, v0), v0);
            else lp_load_aff(Pp, part, e, lane);
            col_entry(Qq, tq, vq);
            fe dinv;
            if (e > 0) {
                fe pr;
                lp_load_fe(pr, pref, e - 1, lane);
                dinv = fmul(inv, pr);
            } else {
                dinv = inv;
            }
            bool special = aff_is_inf(Pp) || aff_is_inf(Qq);
            fe dx;
            if (!special) {
                fe_sub(dx, Qq.x, Pp.x);
                special = fe_is_zero(dx);
            }
            if (!special) {
                inv = fmul(inv, dx);
                fe dy, lam, t0;
                fe_sub(dy, Qq.y, Pp.y);
                lam = fmul(dy, dinv);              // slope
                t0 = fsqr(lam);
                fe_sub(t0, t0, Pp.x);
                fe_sub(R.x, t0, Qq.x);             // x3 = lam^2 - x1 - x2
                fe_sub(t0, Pp.x, R.x);
                t0 = fmul(lam, t0);
                fe_sub(R.y, t0, Pp.y);             // y3 = lam (x1 - x3) - y1
                fe_canon(R.x, R.x);
                fe_canon(R.y, R.y);
            } else {
                jac J;
                jac_from_aff(J, Pp);
                jac_madd(J, Qq);
                if (jac_is_inf(J)) {
                    fe_zero(R.x);
                    fe_zero(R.y);
                } else {
                    fe zi;
                    fe_inv(zi, J.Z);
                    jac_to_aff_with_zinv(R, J, zi);
                }
            }
            lp_store_aff(part, e, lane, R);
        }
    }
    for (int e = 0; e < E; e++) {
        const uint32_t code = P.codes[(size_t)s * a.emax + e];
        uint32_t v1, v0;
        aff R;
        if (comp(code, 1, v1) < 0) col_entry(R, comp(code, 0, v0), v0);   // a single component
        else lp_load_aff(R, part, e, lane);
        store_table(e, R);
    }
}

struct GatherArgs {
    int m, l, lp, njb, emax;
    int s0, nstrips_chunk;
    bool first;
    const uint4* table;
    size_t table_points;
    uint4* ctC;            // Jacobian ciphertext matrix m x l
    int parts;             // warps per output splitting the chunk's strips (1: accumulate into ctC)
    uint4* partial;        // parts > 1: Jacobian partial sums, parts matrices laid out like ctC
};

// Accumulation of one warp item (output row i, component c, 32 columns) over
// the strips of a chunk.  CG = true reads tables and accumulators through L2
// only (ld.global.cg): in the persistent batched kernel they were written by
// other SMs during the same launch.
template <bool CG>
__device__ __forceinline__ void gather_item(const GatherArgs& a, const PlanPtrs& P, long long gw) {
    // Rows innermost: the warps resident at a time cover every row of a few
    // column blocks, so each strip's table region is fetched once per block
    // while those warps walk the strips together.
    // With parts > 1 (small outputs), warp gw / (m 2 njb) takes part p of
    // the chunk's strips and leaves its partial sum for combine_kernel.
    const unsigned lane = threadIdx.x & 31u;
    const long long per_part = (long long)a.m * 2 * a.njb;
    const int part = (int)(gw / per_part);
    gw %= per_part;
    const int i = (int)(gw % a.m);
    const int rem = (int)(gw / a.m);
    const int c = rem / a.njb, jb = rem % a.njb;
    const int j = jb * 32 + (int)lane;
    const size_t ml = (size_t)a.m * a.l;
    uint4* Cc = (a.parts > 1 ? a.partial + (size_t)part * 12 * ml : a.ctC) + (size_t)c * 6 * ml;
    // The running sum is kept as (X, Y, Z^2, Z^3): its mixed additions then
    // cost 8M + 2S, and Z itself is rebuilt once at the end.
    jacz acc;
    if (a.first || a.parts > 1 || j >= a.l) {
        jacz_set_inf(acc);
    } else {
        jac prev;
        if (CG) load_jac_cg(prev, Cc, ml, (size_t)i * a.l + j);
        else load_jac(prev, Cc, ml, (size_t)i * a.l + j);
        jacz_from_jac(acc, prev);
    }
    const uint16_t* rk = P.rank + (size_t)a.s0 * a.m + i;
    aff T;
    const int s_lo = (int)((long long)a.nstrips_chunk * part / a.parts);
    const int s_hi = (int)((long long)a.nstrips_chunk * (part + 1) / a.parts);
    for (int sl = s_lo; sl < s_hi; sl++) {
        const uint16_t code = rk[(size_t)sl * a.m];
        if (code == NO_RANK) continue;
#ifdef PCMM_DEBUG_BOUNDS
        if (code >= P.nent[a.s0 + sl]) {   // a rank past the strip's table
            atomicOr(P.status, DEV_ERR_BOUNDS);
            continue;
        }
#endif
        const size_t ti = (((size_t)sl * a.emax + code) * 2 + c) * a.lp + j;
        if (CG) load_aff_cg(T, a.table, a.table_points, ti);
        else load_aff(T, a.table, a.table_points, ti);
        jacz_madd_t<PCMM_GATHER_INLINE>(acc, T);
    }
    if (j < a.l) {
        jac out;
        jac_from_jacz(out, acc);
        store_jac(Cc, ml, (size_t)i * a.l + j, out);
    }
}

// Expected number of distinct non-zero values when m values are drawn
// uniformly from [0, 2^bits).
inline double expected_distinct_nonzero(int m, int bits) {
    const double V = ldexp(1.0, bits);
    const double present = V * (1.0 - pow(1.0 - 1.0 / V, (double)m));
    const double zero = 1.0 - pow(1.0 - 1.0 / V, (double)m);
    double d = present - zero;
    return d < 0 ? 0 : d;
}

// Modelled time of one PC-MM in field-multiplication units (a squaring
// counted as one) for strip width k.  Gather: one mixed addition (11) per
// row, strip and ciphertext chain with a non-zero code.  Table build: per
// column the level-1 prefix sums (mixed additions) and the level-N
// double-and-add (about 2w operations of 8); the normalisation (5 per entry,
// along the chain's ratios) of the strip table (k = 1) or of the column
// tables (k > 1); for k > 1 the
// tuple entries by affine additions (6 per further non-zero component).  The
// table work is weighted by 1.9, fitted to GB300 timings of the
// 1024 x 1024 x 256 product for every w and k (the table build issues its
// multiplications less efficiently than the gather, and its tuple rounds
// reload their operands from scratch).
inline double model_cost(int m, int n, int l, int w, int k) {
    const double MADD = 11, DBL = 8, NORM = 5, AFF = 6, TABLE_WEIGHT = 1.9;
    const double chains = 2.0 * l;
    const int nstrips = (n + k - 1) / k;
    const double n1 = expected_distinct_nonzero(m, w);
    const double E = k == 1 ? n1 : expected_distinct_nonzero(m, w * k);
    const double nz1 = 1.0 - ldexp(1.0, -w);
    const double col = n * chains * (n1 * MADD + 2.0 * w * DBL);
    const double norm = (k == 1 ? nstrips * E : n * n1) * chains * NORM;
    const double extra = k * nz1 - 1.0;
    const double tup = k > 1 ? nstrips * chains * E * (extra > 0 ? extra : 0.0) * AFF : 0.0;
    const double gather = (double)m * chains * nstrips * (1.0 - ldexp(1.0, -w * k)) * MADD;
    return gather + TABLE_WEIGHT * (col + norm + tup);
}


}  // namespace cussen
}  // namespace pcmm
