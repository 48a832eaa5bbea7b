// Cussen's compression-reconstruction PC-MM (Algorithms 2 and 3) on sm_103a.
//
// Three kernels per pass over a chunk of column strips of A:
//
//  plan   (once per call, one CTA per strip; plaintext only)
//         For every column: level 1 = the distinct non-zero values sorted
//         ascending; for w < N its consecutive differences are sorted and
//         deduplicated into level w + 1, recording for every element of
//         level w its position in level w + 1 (the tracking pointers);
//         level N keeps its values.  A zero contributes the identity and is
//         dropped from every level.  For the strip: the code of every row
//         (its k entries packed w bits apiece), the sorted list of distinct
//         non-zero codes, and each row's rank in that list (0xFFFF for 0).
//  table  (one warp per strip, ciphertext component and 32 output columns)
//         Level N: the compressed values times the ciphertext point B_c^(kj)
//         by double-and-add (the ECSMs of Algorithm 3).  Levels N-1..1: each
//         element of level w is the entry of level w + 1 its tracking pointer
//         names, and a running prefix sum of points turns the multiples of
//         differences into the multiples of the level's sorted values.
//         Level 1 is the per-column table v B_c^(kj) over the distinct values
//         v of the column, a chain of mixed additions in (X, Y, Z^2, Z^3).
//         For strips of k > 1 columns, each distinct k-tuple adds its
//         columns' entries (affine additions, one shared inversion per
//         round).  The tables are normalised to affine coordinates in the
//         same kernel: level 2 by Montgomery's simultaneous inversion, the
//         level-1 chains by walking Z^-2 and Z^-3 back along the factors the
//         chain multiplied them by; the inversion is shared by the lanes of
//         a warp and, when the block's four warps follow one strip's plan,
//         by the whole block.
//  gather (one warp per output row i, component c and 32 output columns)
//         C_ij += T_s[rank_s(i)] for every strip s: the "un-sort and re-insert
//         duplicates" step of Algorithm 2 fused with the accumulation of
//         Algorithm 3, one mixed addition per strip into an accumulator in
//         (X, Y, Z^2, Z^3).  The rank is the same for the whole warp (one
//         broadcast load); the 32 lanes' table entries are adjacent, so the
//         four 16-byte loads per point are coalesced.  Small outputs split
//         their strips over several warps (combine_kernel adds the parts).
#include <cuda_runtime.h>

#include "cussen_core.cuh"
#include "profiler.cuh"

using namespace pcmm;
using namespace pcmm::cussen;

// Minimum resident blocks per SM requested from the compiler (its register
// budget).  Measured on GB300: the gather is pipe-bound (5 blocks at 96
// registers run as fast as 8); the table build waits on its scratch and
// spill traffic, so more resident warps pay despite more spilling: table time
// per headline step 46.3 ms at 4 blocks (128 registers), 45.1 at 5, 45.5 at
// 6, 45.0 at 7 (72 registers), 47.3 at 8; per wide-value step 261.7, 259.3,
// 252.7, 247.1 and 261.9 ms.  Build-time tunables.
#ifndef PCMM_GATHER_MINBLOCKS
#define PCMM_GATHER_MINBLOCKS 5
#endif
#ifndef PCMM_TABLE_MINBLOCKS
#define PCMM_TABLE_MINBLOCKS 7
#endif

namespace {

template <class TA>
__global__ void __launch_bounds__(PLAN_THREADS) plan_kernel(const TA* __restrict__ A, int m, int n, int w,
                                                            int k, PlanPtrs P) {
    plan_strip(A, m, n, w, k, P, blockIdx.x);
}

__global__ void __launch_bounds__(128, PCMM_TABLE_MINBLOCKS) table_kernel(TableArgs a, PlanPtrs P) {
    const long long item = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nitems = (long long)a.nstrips_chunk * 2 * a.njb;
    if (item >= nitems) return;
    table_item(a, P, item, a.scratch + (size_t)item * a.item_u4);
}

__global__ void __launch_bounds__(128, PCMM_GATHER_MINBLOCKS) gather_kernel(GatherArgs a, PlanPtrs P) {
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (long long)a.m * 2 * a.njb * a.parts) return;
    gather_item<false>(a, P, gw);
}

// Adds the parts partial sums of every output point (and, after the first
// pass, the accumulated value) into ctC: one thread per point.
__global__ void __launch_bounds__(128) combine_kernel(const uint4* __restrict__ partial, int parts,
                                                      uint4* __restrict__ ctC, size_t ml, bool first) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * ml) return;
    const size_t c = t / ml, idx = t % ml;
    uint4* Cc = ctC + c * 6 * ml;
    jac acc;
    if (first) jac_set_inf(acc);
    else load_jac(acc, Cc, ml, idx);
    for (int p = 0; p < parts; p++) {
        jac Q;
        load_jac(Q, partial + (size_t)p * 12 * ml + c * 6 * ml, ml, idx);
        jac_add(acc, Q);
    }
    store_jac(Cc, ml, idx, acc);
}

}  // namespace

extern "C" int pcmm_cussen_choose_k(int m, int n, int l, int w) {
    if (m < 1 || n < 1 || l < 1 || w < 1 || w > PCMM_MAX_W16) return 0;
    // A wider strip must win by 3%: its tables and scratch grow with 2^(w k).
    int best = 1;
    double bc = model_cost(m, n, l, w, 1);
    for (int k = 2; w * k <= PCMM_MAX_WK && k <= n; k++) {
        double c = model_cost(m, n, l, w, k);
        if (c < 0.97 * bc) { bc = c; best = k; }
    }
    return best;
}

// Table items (warps) per pass come in whole waves of the table kernel on a
// 152-SM GB300 (PCMM_TABLE_MINBLOCKS blocks of 4 warps per SM), so that only a
// pass's last wave can run partly empty: four waves when one pass's scratch
// and tables fit in PASS_BYTES_CAP, else as many whole waves as fit, at
// least one.  Whole-wave passes measured 3 ms per headline step faster than
// passes of 4096 items (at 4 blocks per SM).
#ifndef PCMM_TARGET_WAVES
#define PCMM_TARGET_WAVES 4
#endif
static const size_t WAVE_ITEMS = 152 * PCMM_TABLE_MINBLOCKS * 4;
static const size_t TARGET_WAVES = PCMM_TARGET_WAVES;
static const size_t PASS_BYTES_CAP = (size_t)16 << 30;

namespace {
size_t default_strips(const Layout& L);
}

namespace {

template <class TA>
pcmm_status launch_plan(const Layout& L, const TA* A, const PlanPtrs& P, cudaStream_t st) {
    if (cudaMemsetAsync(P.status, 0, 4, st) != cudaSuccess) return PCMM_ECUDA;
    {
        ProfScope ps(KID_PLAN, st);
        plan_kernel<TA><<<L.nstrips, PLAN_THREADS, 0, st>>>(A, L.m, L.n, L.w, L.k, P);
    }
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

// Warps per output for the gather of a pass of S strips: when the outputs
// alone give fewer than GATHER_WARPS_TARGET warps (about four waves of the
// gather on 152 SMs), each output's strips are split into up to 32 parts of
// at least 16 strips, and combine_kernel adds the partial sums (one full
// addition per part against at least 16 mixed additions).
const long long GATHER_WARPS_TARGET = 12288;

int gather_parts(const Layout& L, size_t S) {
    const long long warps = (long long)L.m * 2 * L.njb;
    if (warps >= GATHER_WARPS_TARGET) return 1;
    long long parts = (GATHER_WARPS_TARGET + warps - 1) / warps;
    const long long by_strips = (long long)S / 16;
    if (parts > by_strips) parts = by_strips;
    if (parts > 32) parts = 32;
    return parts < 1 ? 1 : (int)parts;
}

size_t partial_bytes(const Layout& L, int parts) {
    return parts > 1 ? align256((size_t)parts * 2 * L.m * L.l * 96) : 0;
}

// Table build and gather over chunks of S strips, using the scratch area at
// `chunk` (S * per_strip_bytes bytes) and, when parts > 1, the partial sums
// at `partial` (partial_bytes(L, parts) bytes).
pcmm_status launch_exec(const Layout& L, const PlanPtrs& P, const uint32_t* ctB, uint32_t* ctC,
                        uint8_t* chunk, size_t S, uint8_t* partial, int parts, cudaStream_t st) {
    uint4* scratch = (uint4*)chunk;
    uint4* table = (uint4*)(chunk + align256(S * L.items_per_strip * L.item_u4 * 16));
    const size_t ml = (size_t)L.m * L.l;
    for (int s0 = 0; s0 < L.nstrips; s0 += (int)S) {
        const int sc = (int)((size_t)(L.nstrips - s0) < S ? (size_t)(L.nstrips - s0) : S);
        TableArgs ta;
        ta.ctB = (const uint4*)ctB;
        ta.m = L.m; ta.n = L.n; ta.l = L.l; ta.w = L.w; ta.k = L.k;
        ta.lp = L.lp; ta.njb = L.njb; ta.n1max = L.n1max; ta.l2max = L.l2max; ta.emax = L.emax;
        ta.s0 = s0; ta.nstrips_chunk = sc;
        ta.scratch = scratch;
        ta.item_u4 = L.item_u4;
        ta.table = table;
        ta.table_points = S * L.table_points_per_strip;
        // Four consecutive items (one 128-thread block) belong to one strip
        // exactly when a strip has a multiple of 4 items; then every block is
        // full and its warps follow the same plan, and share inversions.
        ta.bshare = (L.items_per_strip % 4) == 0;
        const long long items = (long long)sc * L.items_per_strip;
        {
            ProfScope ps(KID_TABLE, st);
            table_kernel<<<(unsigned)((items + 3) / 4), 128, 0, st>>>(ta, P);
        }
        PCMM_CUDA_CHECK_LAUNCH();
        GatherArgs ga;
        ga.m = L.m; ga.l = L.l; ga.lp = L.lp; ga.njb = L.njb; ga.emax = L.emax;
        ga.s0 = s0; ga.nstrips_chunk = sc;
        ga.first = (s0 == 0);
        ga.table = table;
        ga.table_points = ta.table_points;
        ga.ctC = (uint4*)ctC;
        // A short last chunk may take fewer parts than the buffer holds.
        const int pc = parts > 1 ? (sc / 16 < parts ? (sc / 16 > 1 ? sc / 16 : 1) : parts) : 1;
        ga.parts = pc;
        ga.partial = (uint4*)partial;
        const long long warps = (long long)L.m * 2 * L.njb * pc;
        {
            ProfScope ps(KID_GATHER, st);
            gather_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(ga, P);
        }
        PCMM_CUDA_CHECK_LAUNCH();
        if (pc > 1) {
            ProfScope ps(KID_COMBINE, st);
            combine_kernel<<<(unsigned)((2 * ml + 127) / 128), 128, 0, st>>>((const uint4*)partial, pc,
                                                                           (uint4*)ctC, ml, s0 == 0);
        }
        PCMM_CUDA_CHECK_LAUNCH();
    }
    return PCMM_OK;
}

size_t default_strips(const Layout& L) {
    const size_t ips = L.items_per_strip;
    const size_t cap = PASS_BYTES_CAP / L.per_strip_bytes;   // strips within the byte cap
    size_t waves = TARGET_WAVES;
    while (waves > 1 && waves * WAVE_ITEMS / ips > cap) waves--;
    size_t S = waves * WAVE_ITEMS / ips;                      // whole strips within the waves
    if (S > (size_t)L.nstrips) S = L.nstrips;
    return S < 1 ? 1 : S;
}

// Bytes of execution workspace (beyond the plan) the default configuration
// uses: the gather's partial sums, then passes of default_strips strips.
size_t default_exec_bytes(const Layout& L) {
    const size_t S = default_strips(L);
    return partial_bytes(L, gather_parts(L, S)) + S * L.per_strip_bytes;
}

// Splits `avail` bytes of execution workspace into the partial sums (when
// the gather splits its strips) and passes of S strips; the partial sums are
// dropped when both do not fit.  False when not even one strip fits.
bool exec_space(const Layout& L, size_t avail, size_t& S, int& parts, size_t& pbytes) {
    parts = gather_parts(L, default_strips(L));
    pbytes = partial_bytes(L, parts);
    if (parts > 1 && avail >= pbytes + L.per_strip_bytes) {
        S = (avail - pbytes) / L.per_strip_bytes;
    } else {
        parts = 1;
        pbytes = 0;
        if (avail < L.per_strip_bytes) return false;
        S = avail / L.per_strip_bytes;
    }
    if (S > (size_t)L.nstrips) S = L.nstrips;
    const int ps = gather_parts(L, S);
    if (ps < parts) parts = ps;
    return true;
}

}  // namespace

namespace {

template <class TA>
pcmm_status cussen_call(const TA* A, int m, int n, int w, const uint32_t* ctB, int l, uint32_t* ctC, int k,
                        void* ws, size_t ws_bytes, pcmm_stream_t stream) {
    if (!A || !ctB || !ctC || !ws || ((uintptr_t)ws & 255u)) return PCMM_EINVAL;
    if (m < 1 || n < 1 || l < 1 || w < 1 || w > 8 * (int)sizeof(TA)) return PCMM_EINVAL;
    if (k == 0) k = pcmm_cussen_choose_k(m, n, l, w);
    Layout L;
    if (!make_layout(L, m, n, l, w, k)) return PCMM_EINVAL;
    if (ws_bytes < L.plan_bytes) return PCMM_ENOMEM;
    size_t S, pbytes;
    int parts;
    if (!exec_space(L, ws_bytes - L.plan_bytes, S, parts, pbytes)) return PCMM_ENOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    PlanPtrs P = plan_ptrs(L, ws);
    pcmm_status rc = launch_plan(L, A, P, st);
    if (rc != PCMM_OK) return rc;
    uint8_t* partial = (uint8_t*)ws + L.plan_bytes;
    return launch_exec(L, P, ctB, ctC, partial + pbytes, S, partial, parts, st);
}

}  // namespace

extern "C" size_t pcmm_cussen_workspace_bytes_for(int m, int n, int l, int w, int k, int strips) {
    Layout L;
    if (k < 1 || strips < 1 || !make_layout(L, m, n, l, w, k)) return 0;
    const size_t S = (size_t)strips < (size_t)L.nstrips ? (size_t)strips : (size_t)L.nstrips;
    // Room for the gather's partial sums as the default pass sizes them
    // (exec_space reserves them first, then fits the strips).
    return L.plan_bytes + partial_bytes(L, gather_parts(L, default_strips(L))) + S * L.per_strip_bytes;
}

extern "C" size_t pcmm_cussen_workspace_bytes(int m, int n, int l, int w, int k) {
    if (k == 0) k = pcmm_cussen_choose_k(m, n, l, w);
    Layout L;
    if (!make_layout(L, m, n, l, w, k)) return 0;
    return L.plan_bytes + default_exec_bytes(L);
}

extern "C" size_t pcmm_workspace_bytes(int op, int m, int n, int l, int w, int k) {
    const bool shape_ok = m >= 1 && n >= 1 && l >= 1 && w >= 1 && w <= PCMM_MAX_W16;
    size_t b = 0;
    switch (op) {
        case PCMM_OP_ENCRYPT:
            return pcmm_encrypt_workspace_bytes();
        case PCMM_OP_SCHOOLBOOK:
        case PCMM_OP_NORMALIZE:
            return shape_ok ? 0 : PCMM_WS_INVALID;
        case PCMM_OP_CUSSEN:
            b = pcmm_cussen_workspace_bytes(m, n, l, w, k);
            break;
        case PCMM_OP_CUSSEN_PLAN:
            b = pcmm_cussen_plan_bytes(m, n, w, k ? k : pcmm_cussen_choose_k(m, n, l, w));
            break;
        case PCMM_OP_CUSSEN_EXEC:
            b = pcmm_cussen_exec_bytes(m, n, l, w, k ? k : pcmm_cussen_choose_k(m, n, l, w));
            break;
        case PCMM_OP_STRASSEN:
            b = pcmm_strassen_workspace_bytes(m, n, l, w, k);
            break;
        default:
            return PCMM_WS_INVALID;
    }
    return (shape_ok && b) ? b : PCMM_WS_INVALID;
}

extern "C" pcmm_status pcmm_cussen(const uint8_t* A, int m, int n, int w, const uint32_t* ctB, int l,
                                   uint32_t* ctC, int k, void* ws, size_t ws_bytes,
                                   pcmm_stream_t stream) {
    return cussen_call(A, m, n, w, ctB, l, ctC, k, ws, ws_bytes, stream);
}

extern "C" pcmm_status pcmm_cussen16(const uint16_t* A, int m, int n, int w, const uint32_t* ctB, int l,
                                     uint32_t* ctC, int k, void* ws, size_t ws_bytes,
                                     pcmm_stream_t stream) {
    return cussen_call(A, m, n, w, ctB, l, ctC, k, ws, ws_bytes, stream);
}

extern "C" size_t pcmm_cussen_plan_bytes(int m, int n, int w, int k) {
    Layout L;
    if (!make_layout(L, m, n, 1, w, k)) return 0;
    return L.plan_bytes;
}

extern "C" pcmm_status pcmm_cussen_plan(const uint8_t* A, int m, int n, int w, int k, void* plan,
                                        size_t plan_bytes, pcmm_stream_t stream) {
    if (!A || !plan || ((uintptr_t)plan & 255u) || w > PCMM_MAX_W) return PCMM_EINVAL;
    Layout L;
    if (!make_layout(L, m, n, 1, w, k)) return PCMM_EINVAL;
    if (plan_bytes < L.plan_bytes) return PCMM_ENOMEM;
    return launch_plan(L, A, plan_ptrs(L, plan), (cudaStream_t)stream);
}

extern "C" size_t pcmm_cussen_exec_bytes(int m, int n, int l, int w, int k) {
    Layout L;
    if (!make_layout(L, m, n, l, w, k)) return 0;
    return default_exec_bytes(L);
}

extern "C" pcmm_status pcmm_cussen_execute(const void* plan, int m, int n, int w, int k,
                                           const uint32_t* ctB, int l, uint32_t* ctC, void* ws,
                                           size_t ws_bytes, pcmm_stream_t stream) {
    if (!plan || !ctB || !ctC || !ws || ((uintptr_t)plan & 255u) || ((uintptr_t)ws & 255u))
        return PCMM_EINVAL;
    Layout L;
    if (!make_layout(L, m, n, l, w, k)) return PCMM_EINVAL;
    size_t S, pbytes;
    int parts;
    if (!exec_space(L, ws_bytes, S, parts, pbytes)) return PCMM_ENOMEM;
    return launch_exec(L, plan_ptrs(L, const_cast<void*>(plan)), ctB, ctC, (uint8_t*)ws + pbytes, S,
                       (uint8_t*)ws, parts, (cudaStream_t)stream);
}

extern "C" pcmm_status pcmm_workspace_status(const void* ws, uint32_t* status_host, pcmm_stream_t stream) {
    if (!ws || !status_host) return PCMM_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return PCMM_ECUDA;
    if (cudaMemcpy(status_host, ws, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return PCMM_ECUDA;
    return PCMM_OK;
}
