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
constexpr uint16_t NO_RANK = 0xFFFFu;
constexpr int PLAN_THREADS = 256;

struct Layout {
    int m, n, l, w, k;
    int nstrips, n1max, l2max, emax, lp, njb;
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

inline bool make_layout(Layout& L, int m, int n, int l, int w, int k) {
    if (m < 1 || n < 1 || l < 1 || w < 1 || w > PCMM_MAX_W || k < 1 || w * k > PCMM_MAX_WK) return false;
    L.m = m; L.n = n; L.l = l; L.w = w; L.k = k;
    L.nstrips = (n + k - 1) / k;
    L.n1max = (1 << w) - 1 < m ? (1 << w) - 1 : m;
    L.l2max = level2_bound(w);
    L.emax = (1 << (w * k)) - 1 < m ? (1 << (w * k)) - 1 : m;
    L.njb = (l + 31) / 32;
    L.lp = L.njb * 32;
    size_t off = 256;  // status word and padding
    L.off_rank = off;  off = align256(off + (size_t)L.nstrips * m * 2);
    L.off_nent = off;  off = align256(off + (size_t)L.nstrips * 4);
    L.off_codes = off; off = align256(off + (size_t)L.nstrips * L.emax * 2);
    L.off_len = off;   off = align256(off + (size_t)n * NLEV * 2);
    L.off_vN = off;    off = align256(off + (size_t)n * 256);
    L.off_ptr = off;   off = align256(off + (size_t)n * (NLEV > 1 ? NLEV - 1 : 1) * 256);
    L.off_rank1 = off; off = align256(off + (size_t)n * 256);
    L.plan_bytes = off;
    // Per warp item (lane-planar): Jacobian column table and level ping-pong,
    // affine level-2 entries, affine column tables and Jacobian tuples (k > 1),
    // prefix products for the normalisations.
    const size_t jac_ents = (size_t)L.n1max + 2 * (size_t)L.l2max + (k > 1 ? (size_t)L.emax : 0);
    const size_t aff_ents = (size_t)L.l2max + (k > 1 ? (size_t)k * L.n1max : 0);
    L.item_u4 = jac_ents * 6 * 32 + aff_ents * 4 * 32 + (size_t)L.emax * 2 * 32;
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
    uint8_t* col_vN;
    uint8_t* col_ptr;
    uint8_t* col_rank1;
};

inline PlanPtrs plan_ptrs(const Layout& L, void* ws) {
    uint8_t* b = (uint8_t*)ws;
    PlanPtrs P;
    P.status = (uint32_t*)b;
    P.rank = (uint16_t*)(b + L.off_rank);
    P.nent = (int32_t*)(b + L.off_nent);
    P.codes = (uint16_t*)(b + L.off_codes);
    P.col_len = (uint16_t*)(b + L.off_len);
    P.col_vN = b + L.off_vN;
    P.col_ptr = b + L.off_ptr;
    P.col_rank1 = b + L.off_rank1;
    return P;
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

// Block-level plan of strip s (all PLAN_THREADS threads of the block call).
__device__ __forceinline__ void plan_strip(const uint8_t* __restrict__ A, int m, int n, int w, int k,
                                           int emax, const PlanPtrs& P, int s) {
    __shared__ uint32_t spres[128];
    __shared__ uint32_t spref[128];
    __shared__ uint32_t wbm[PLAN_THREADS / 32][8];
    __shared__ uint16_t wlev[PLAN_THREADS / 32][2][256];
    __shared__ uint8_t wpos[PLAN_THREADS / 32][256];
    const int c0 = s * k;
    const int kw = (c0 + k <= n) ? k : n - c0;
    const uint32_t amask = (1u << w) - 1u;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;

    // ---- per-column compression levels (one warp per column) ----
    for (int t = (int)warp; t < kw; t += PLAN_THREADS / 32) {
        const int col = c0 + t;
        uint32_t* bm = wbm[warp];
        uint8_t* pos = wpos[warp];
        if (lane < 8) bm[lane] = 0u;
        __syncwarp();
        bool bad = false;
        for (int i = (int)lane; i < m; i += 32) {
            uint32_t v = A[(size_t)i * n + col];
            bad |= v > amask;
            v &= amask;
            if (v) atomicOr(&bm[v >> 5], 1u << (v & 31u));
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(P.status, DEV_ERR_A_RANGE);
        __syncwarp();
        uint16_t* cur = wlev[warp][0];
        uint16_t* nxt = wlev[warp][1];
        int len = extract_sorted(bm, cur, pos);
        // value -> level-1 position, for the k-tuple assembly
        for (int v = (int)lane; v < 256; v += 32) {
            const bool present = v > 0 && ((bm[v >> 5] >> (v & 31)) & 1u);
            P.col_rank1[(size_t)col * 256 + v] = present ? pos[v] : (uint8_t)0xff;
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
            for (int e = (int)lane; e < len; e += 32) {
                const int d = (int)cur[e] - (e ? (int)cur[e - 1] : 0);
                P.col_ptr[((size_t)col * (NLEV - 1) + (lev - 1)) * 256 + e] = pos[d];
            }
            if (lane == 0) P.col_len[(size_t)col * NLEV + lev] = (uint16_t)nlen;
            __syncwarp();
            uint16_t* tmp = cur; cur = nxt; nxt = tmp;
            len = nlen;
        }
        for (int e = (int)lane; e < len; e += 32) P.col_vN[(size_t)col * 256 + e] = (uint8_t)cur[e];
        __syncwarp();
    }

    // ---- strip codes, distinct codes and per-row ranks (whole block) ----
    for (int x = threadIdx.x; x < 128; x += blockDim.x) spres[x] = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        uint32_t code = 0;
        for (int t = 0; t < kw; t++) code |= ((uint32_t)A[(size_t)i * n + c0 + t] & amask) << (w * t);
        if (code) atomicOr(&spres[code >> 5], 1u << (code & 31u));
    }
    __syncthreads();
    if (warp == 0) {
        int cnt = 0;
        for (int q = 0; q < 4; q++) cnt += __popc(spres[lane * 4 + q]);
        int total;
        int base = warp_excl_scan(cnt, total);
        for (int q = 0; q < 4; q++) {
            spref[lane * 4 + q] = (uint32_t)base;
            base += __popc(spres[lane * 4 + q]);
        }
        if (lane == 0) P.nent[s] = total;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        uint32_t code = 0;
        for (int t = 0; t < kw; t++) code |= ((uint32_t)A[(size_t)i * n + c0 + t] & amask) << (w * t);
        uint16_t r = NO_RANK;
        if (code) r = (uint16_t)(spref[code >> 5] + __popc(spres[code >> 5] & ((1u << (code & 31u)) - 1u)));
        P.rank[(size_t)s * m + i] = r;
    }
    if (k > 1) {
        for (int wd = threadIdx.x; wd < 128; wd += blockDim.x) {
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
}

struct TableArgs {
    const uint4* ctB;      // affine ciphertext matrix n x l
    const uint8_t* A;
    int m, n, l, w, k, lp, njb, n1max, l2max, emax;
    int s0, nstrips_chunk;
    uint4* scratch;        // lane-planar per-item scratch
    size_t item_u4;
    uint4* table;          // affine, quad-planar, table_points points
    size_t table_points;
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

__device__ __forceinline__ bool fe_is_one(const fe& a) {
    uint32_t z = (a.v[0] ^ 1u) | a.v[1] | a.v[2] | a.v[3] | a.v[4] | a.v[5] | a.v[6] | a.v[7];
    return z == 0u;
}

// Normalises E lane-planar Jacobian entries to canonical affine (infinity ->
// (0, 0)) and hands entry e to store(e, point).  Montgomery's simultaneous
// inversion: per-lane prefix products of the Z's (kept in pref), then one
// warp-wide inversion.  When every Z in the warp is already 1 the entries
// are copied without any inversion.  All 32 lanes call with the same E.
template <class Store>
__device__ __forceinline__ void lp_normalize(const uint4* src, int E, uint4* pref, unsigned lane,
                                             Store store) {
    if (E <= 0) return;
    bool ones = true;
    fe acc;
    fe_one(acc);
    for (int e = 0; e < E; e++) {
        fe z;
        lp_load_z(z, src, e, lane);
        ones &= fe_is_one(z);
        if (fe_is_zero(z)) fe_one(z);
        acc = fmul(acc, z);
        lp_store_fe(pref, e, lane, acc);
    }
    if (__all_sync(0xffffffffu, ones)) {
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
    warp_inverse(inv, acc);
    for (int e = E - 1; e >= 0; e--) {
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
    uint4* ents_x = levB + (size_t)a.l2max * 192;                         // emax Jacobian (k > 1)
    uint4* l2aff = ents_x + (a.k > 1 ? (size_t)a.emax * 192 : 0);         // l2max affine
    uint4* colaff = l2aff + (size_t)a.l2max * 128;                        // k * n1max affine (k > 1)
    uint4* pref = colaff + (a.k > 1 ? (size_t)a.k * a.n1max * 128 : 0);   // emax field elements

    const int E = P.nent[s];
    const size_t tbase = (size_t)s_local * a.emax;
    auto store_table = [&](int e, const aff& q) {
        store_aff(a.table, a.table_points, ((tbase + e) * 2 + c) * a.lp + j, q);
    };
    bool bad = false;

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
        if (bad) break;
        // Level N: multiples of the compressed values (double-and-add).
        uint4* src = levA;
        for (int e = 0; e < lens[NLEV - 1]; e++) {
            jac T;
            jac_mul_small(T, Pb, P.col_vN[(size_t)col * 256 + e]);
            lp_store_jac(src, e, lane, T);
        }
        uint4* alt = levB;
        // Levels N-1..2: un-sort by the tracking pointers, then prefix sums.
        for (int lev = NLEV - 1; lev >= 2; lev--) {
            const uint8_t* ptr = P.col_ptr + ((size_t)col * (NLEV - 1) + (lev - 1)) * 256;
            jac acc, D;
            jac_set_inf(acc);
            for (int e = 0; e < lens[lev - 1]; e++) {
                lp_load_jac(D, src, ptr[e], lane);
                jac_add(acc, D);
                lp_store_jac(alt, e, lane, acc);
            }
            uint4* tmp = src; src = alt; alt = tmp;
        }
        // Level 2 (multiples of the level-1 differences) to affine, so that
        // the level-1 prefix sums are mixed additions.
        lp_normalize(src, lens[1], pref, lane, [&](int e, const aff& q) { lp_store_aff(l2aff, e, lane, q); });
        // Level 1: the multiples of the column's sorted distinct values.
        {
            const uint8_t* ptr = P.col_ptr + (size_t)col * (NLEV - 1) * 256;
            jac acc;
            aff D;
            jac_set_inf(acc);
            for (int e = 0; e < lens[0]; e++) {
                lp_load_aff(D, l2aff, ptr[e], lane);
                jac_madd(acc, D);
                lp_store_jac(coltab, e, lane, acc);
            }
        }
        if (a.k == 1) {
            // The column table is the strip table.
            lp_normalize(coltab, E, pref, lane, store_table);
            return;
        }
        uint4* ca = colaff + (size_t)t * a.n1max * 128;
        lp_normalize(coltab, lens[0], pref, lane, [&](int e, const aff& q) { lp_store_aff(ca, e, lane, q); });
    }
    if (bad) {
        if (lane == 0) atomicOr(P.status, DEV_ERR_PLAN);
        return;
    }
    // k > 1: one entry per distinct k-tuple, the sum of its columns' (affine)
    // entries, computed in affine coordinates one addition round at a time:
    // round r adds the (r+1)-th non-zero component of every tuple that has
    // one.  The additions of a round are independent, so their slopes share
    // one simultaneous inversion (per-lane prefix products of the x
    // differences, then one warp-wide inversion): about 5M + 1S per entry
    // instead of a mixed addition and a normalisation.  Pairs the affine
    // formula cannot take (infinity, equal or opposite points) use the
    // complete Jacobian addition and their own inversion on a rare branch.
    uint4* part = ents_x;   // affine partial sums (4 quads per entry)
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
        warp_inverse(inv, acc);
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
    const unsigned lane = threadIdx.x & 31u;
    const int i = (int)(gw % a.m);
    const int rem = (int)(gw / a.m);
    const int c = rem / a.njb, jb = rem % a.njb;
    const int j = jb * 32 + (int)lane;
    const size_t ml = (size_t)a.m * a.l;
    uint4* Cc = a.ctC + (size_t)c * 6 * ml;
    jac acc;
    if (a.first || j >= a.l) jac_set_inf(acc);
    else if (CG) load_jac_cg(acc, Cc, ml, (size_t)i * a.l + j);
    else load_jac(acc, Cc, ml, (size_t)i * a.l + j);
    const uint16_t* rk = P.rank + (size_t)a.s0 * a.m + i;
    aff T;
    for (int sl = 0; sl < a.nstrips_chunk; sl++) {
        const uint16_t code = rk[(size_t)sl * a.m];
        if (code == NO_RANK) continue;
        const size_t ti = (((size_t)sl * a.emax + code) * 2 + c) * a.lp + j;
        if (CG) load_aff_cg(T, a.table, a.table_points, ti);
        else load_aff(T, a.table, a.table_points, ti);
        jac_madd(acc, T);
    }
    if (j < a.l) store_jac(Cc, ml, (size_t)i * a.l + j, acc);
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

// Modelled work in field multiplications (a squaring counted as one).
inline double model_cost(int m, int n, int l, int w, int k) {
    const double MADD = 11, ADD = 16, DBL = 8, NORM = 7;
    const double chains = 2.0 * l;
    const int nstrips = (n + k - 1) / k;
    const double n1 = expected_distinct_nonzero(m, w);
    const double E = k == 1 ? n1 : expected_distinct_nonzero(m, w * k);
    double col = n * chains * (n1 * ADD + 2.0 * w * DBL);
    double tup = k > 1 ? nstrips * chains * E * (k - 1) * ADD : 0.0;
    double norm = nstrips * chains * E * NORM;
    double nz = 1.0 - ldexp(1.0, -w * k);
    double gather = (double)m * chains * nstrips * nz * MADD;
    return col + tup + norm + gather;
}


}  // namespace cussen
}  // namespace pcmm
