// Many Cussen PC-MM instances of uneven shapes and bit-widths in one
// persistent launch.
//
// pcmm_batched_prepare (host) sizes every instance (strip width k from the
// caller or the cost model; S strips per pass), lays out the workspace and
// uploads the instance descriptors and the schedule.  pcmm_batched_run then
// enqueues only fixed-size work: two memsets, the plans of all instances
// (one launch, one block per strip) and ONE persistent kernel, so it can be
// captured in a CUDA graph and replayed.
//
// The persistent kernel's blocks pull four tasks at a time (one per warp)
// from a device-wide queue (an atomic counter); when a strip's table tasks
// come in multiples of four, the block's warps build one strip together and
// share each field inversion.  The schedule is a list of segments in round
// order (each padded to a multiple of four tasks): in
// round r, the table-build tasks of every instance's r-th pass of strips,
// then the gather tasks of those passes.  A task may wait (bounded spin) only
// on tasks earlier in the queue:
//   * a gather task of pass r waits for all table tasks of that pass and for
//     all gather tasks of pass r - 1 (they update the same outputs);
//   * a table task of pass r waits for all gather tasks of pass r - 2 (the
//     two table buffers of an instance alternate between passes).
// Every task a block waits on was pulled earlier by a block that is running
// and only waits on even earlier tasks, so the queue always progresses.  A
// wait that exceeds its bound (about one second) sets a status bit and the
// blocks stop pulling tasks instead of hanging.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "cussen_core.cuh"
#include "profiler.cuh"

using namespace pcmm;
using namespace pcmm::cussen;

namespace {

constexpr int TASK_TABLE = 0, TASK_GATHER = 1;
constexpr int BATCH_THREADS = 128;
constexpr int BLOCK_TASKS = BATCH_THREADS / 32;   // tasks a block takes at once, one per warp

struct Inst {
    const uint4* ctB;
    uint4* ctC;
    const uint8_t* A;
    PlanPtrs P;
    uint4* tables;              // two buffers of 4 * table_points uint4
    size_t table_points;        // points per buffer (S strips)
    size_t item_u4;
    int m, n, l, w, k;
    int nstrips, n1max, l2max, emax, lp, njb;
    int S, nchunks;
    int ctr_base;               // 2 counters per pass: tables done, gathers done
};

struct Segment {
    long long start;            // first task index of the segment
    int type, inst, chunk, count;
};

struct BatchHeader {            // device copy, first bytes of the workspace
    uint32_t status;
    int head;                   // next task index
};

__global__ void __launch_bounds__(PLAN_THREADS) batched_plan_kernel(const Inst* __restrict__ insts,
                                                                    const int2* __restrict__ strip_map) {
    const int2 is = strip_map[blockIdx.x];
    const Inst& I = insts[is.x];
    plan_strip(I.A, I.m, I.n, I.w, I.k, I.P, is.y);
}

// Resident blocks per SM requested from the compiler: 4 (128 registers, some
// spilled) measured 1256.9 ms for the 64-instance batch against 1497.9 ms
// uncapped (168 registers, 3 blocks) and 1262.7 ms at 5 blocks.
#ifndef PCMM_BATCH_MINBLOCKS
#define PCMM_BATCH_MINBLOCKS 4
#endif
__global__ void __launch_bounds__(BATCH_THREADS, PCMM_BATCH_MINBLOCKS) batched_kernel(const Inst* __restrict__ insts,
                                                                const Segment* __restrict__ segs, int nsegs,
                                                                long long ntasks, BatchHeader* hdr,
                                                                int* ctrs, uint4* scratch,
                                                                size_t scratch_u4) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const long long warp_id = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint4* my_scratch = scratch + (size_t)warp_id * scratch_u4;
    __shared__ long long sh_t;
    __shared__ int sh_seg, sh_go;
    for (;;) {
        // The block takes BLOCK_TASKS consecutive tasks of one segment (every
        // segment starts at a multiple of BLOCK_TASKS), one per warp.  Every
        // decision below that leads to a barrier or out of the loop is made
        // by thread 0 and read from shared memory, so it is block-uniform.
        if (threadIdx.x == 0) {
            const long long t0 = atomicAdd(&hdr->head, BLOCK_TASKS);
            int go = t0 < ntasks && !(*(volatile uint32_t*)&hdr->status & DEV_ERR_TIMEOUT);
            int lo = 0;
            if (go) {
                // Segment holding task t0 (segments are sorted by start).
                int hi = nsegs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (segs[mid].start <= t0) lo = mid; else hi = mid - 1;
                }
                // Wait (bounded) for the tasks this segment depends on.
                const Segment& sg = segs[lo];
                const Inst& I = insts[sg.inst];
                int* tdone = ctrs + I.ctr_base + 2 * sg.chunk;
                const int sc = min(I.S, I.nstrips - sg.chunk * I.S);
                if (sg.type == TASK_TABLE) {
                    if (sg.chunk >= 2) go = wait_at_least(tdone - 4 + 1, I.m * 2 * I.njb, &hdr->status);
                } else {
                    go = wait_at_least(tdone, sc * 2 * I.njb, &hdr->status);
                    if (go && sg.chunk > 0) go = wait_at_least(tdone - 2 + 1, I.m * 2 * I.njb, &hdr->status);
                }
            }
            sh_t = t0;
            sh_seg = lo;
            sh_go = go;
        }
        __syncthreads();
        const long long t0 = sh_t;
        const int go = sh_go;
        const Segment sg = segs[sh_seg];
        __syncthreads();                      // shared values read before the next round
        if (!go) break;
        const long long item = t0 + warp - sg.start;
        const bool real = item < sg.count;
        const Inst& I = insts[sg.inst];
        const int s0 = sg.chunk * I.S;
        const int sc = min(I.S, I.nstrips - s0);
        uint4* tbuf = I.tables + (size_t)(sg.chunk & 1) * 4 * I.table_points;
        int* tdone = ctrs + I.ctr_base + 2 * sg.chunk;
        if (sg.type == TASK_TABLE) {
            // A strip's items come in multiples of BLOCK_TASKS exactly when
            // its item count is one; then the block's four items belong to one
            // strip, follow one plan and share each inversion.
            const int ips = 2 * I.njb;
            const bool shared = (ips % BLOCK_TASKS) == 0;
            if (real) {
                TableArgs ta;
                ta.ctB = I.ctB;
                ta.bshare = shared;
                ta.m = I.m; ta.n = I.n; ta.l = I.l; ta.w = I.w; ta.k = I.k;
                ta.lp = I.lp; ta.njb = I.njb; ta.n1max = I.n1max; ta.l2max = I.l2max; ta.emax = I.emax;
                ta.s0 = s0; ta.nstrips_chunk = sc;
                ta.scratch = my_scratch;
                ta.item_u4 = I.item_u4;
                ta.table = tbuf;
                ta.table_points = I.table_points;
                table_item(ta, I.P, item, my_scratch);
            }
        } else if (real) {
            GatherArgs ga;
            ga.m = I.m; ga.l = I.l; ga.lp = I.lp; ga.njb = I.njb; ga.emax = I.emax;
            ga.parts = 1; ga.partial = nullptr;
            ga.s0 = s0; ga.nstrips_chunk = sc;
            ga.first = (sg.chunk == 0);
            ga.table = tbuf;
            ga.table_points = I.table_points;
            ga.ctC = I.ctC;
            gather_item<true>(ga, I.P, item);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long left = sg.count - (t0 - sg.start);
            const int done = (int)(left < BLOCK_TASKS ? left : BLOCK_TASKS);
            atomicAdd(tdone + (sg.type == TASK_TABLE ? 0 : 1), done);
        }
    }
}

struct HostLayout {
    std::vector<Inst> insts;
    std::vector<Segment> segs;
    std::vector<int2> strip_map;
    long long ntasks = 0;
    size_t off_insts = 0, off_segs = 0, off_map = 0, off_ctrs = 0, off_scratch = 0, bytes = 0;
    int nctrs = 0;
    size_t scratch_u4 = 0;
    int grid = 0;
};

// Strips per pass of one instance.  An instance's passes run one after
// another, so a pass should hold enough table warps to keep the queue busy
// (PASS_ITEMS) while its two table buffers stay within 2 x BUFFER_CAP bytes:
// at least min(64 strips, 256 MB for both buffers), raised to PASS_ITEMS
// table items, capped by BUFFER_CAP per buffer and by max_strips when given.
// The 64-instance batch measured 1172.4 ms at 1024 items, 1146.3 ms at 2048
// and 1152.5 ms at 4096.
#ifndef PCMM_BATCH_PASS_ITEMS
#define PCMM_BATCH_PASS_ITEMS 2048
#endif
const size_t PASS_ITEMS = PCMM_BATCH_PASS_ITEMS;
const size_t BUFFER_CAP = (size_t)2 << 30;

int strips_per_pass(const Layout& L, int max_strips, int strips) {
    if (strips > 0) {
        size_t S = (size_t)strips;
        const size_t per_strip = align256(L.table_points_per_strip * 64);
        if (S > BUFFER_CAP / per_strip) S = BUFFER_CAP / per_strip;
        if (max_strips > 0 && S > (size_t)max_strips) S = max_strips;
        if (S > (size_t)L.nstrips) S = L.nstrips;
        return S < 1 ? 1 : (int)S;
    }
    const size_t per_strip = align256(L.table_points_per_strip * 64);
    size_t S = ((size_t)256 << 20) / (2 * per_strip);
    if (S > 64) S = 64;
    const size_t by_items = (PASS_ITEMS + L.items_per_strip - 1) / L.items_per_strip;
    if (S < by_items) S = by_items;
    if (S > BUFFER_CAP / per_strip) S = BUFFER_CAP / per_strip;
    if (max_strips > 0 && S > (size_t)max_strips) S = max_strips;
    if (S > (size_t)L.nstrips) S = L.nstrips;
    return S < 1 ? 1 : (int)S;
}

pcmm_status build_layout(const pcmm_problem* probs, int count, int max_strips, int grid,
                         HostLayout& H) {
    if (!probs || count < 1 || grid < 1 || max_strips < 0) return PCMM_EINVAL;
    H = HostLayout();
    H.grid = grid;
    std::vector<Layout> Ls(count);
    size_t off = 256;
    for (int i = 0; i < count; i++) {
        const pcmm_problem& p = probs[i];
        if (!p.A || !p.ctB || !p.ctC || p.w > PCMM_MAX_W || p.strips < 0) return PCMM_EINVAL;
        int k = p.k ? p.k : pcmm_cussen_choose_k(p.m, p.n, p.l, p.w);
        if (!make_layout(Ls[i], p.m, p.n, p.l, p.w, k)) return PCMM_EINVAL;
    }
    // Plans.
    std::vector<size_t> plan_off(count);
    for (int i = 0; i < count; i++) {
        plan_off[i] = off;
        off = align256(off + Ls[i].plan_bytes);
    }
    // Table buffers (two per instance).
    std::vector<size_t> tab_off(count);
    H.insts.resize(count);
    int ctr = 0;
    for (int i = 0; i < count; i++) {
        const Layout& L = Ls[i];
        Inst& I = H.insts[i];
        I.S = strips_per_pass(L, max_strips, probs[i].strips);
        I.nchunks = (L.nstrips + I.S - 1) / I.S;
        I.table_points = (size_t)I.S * L.table_points_per_strip;
        tab_off[i] = off;
        off = align256(off + 2 * I.table_points * 64);
        I.ctr_base = ctr;
        ctr += 2 * I.nchunks;
        I.m = L.m; I.n = L.n; I.l = L.l; I.w = L.w; I.k = L.k;
        I.nstrips = L.nstrips; I.n1max = L.n1max; I.l2max = L.l2max; I.emax = L.emax;
        I.lp = L.lp; I.njb = L.njb; I.item_u4 = L.item_u4;
        H.scratch_u4 = std::max(H.scratch_u4, L.item_u4);
    }
    H.nctrs = ctr;
    // Schedule: rounds of passes; within a round, larger instances first.
    int rounds = 0;
    for (auto& I : H.insts) rounds = std::max(rounds, I.nchunks);
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        const double wa = (double)H.insts[a].m * H.insts[a].l * H.insts[a].nstrips;
        const double wb = (double)H.insts[b].m * H.insts[b].l * H.insts[b].nstrips;
        return wa > wb;
    });
    long long t = 0;
    for (int r = 0; r < rounds; r++) {
        for (int ph = 0; ph < 2; ph++) {
            for (int i : order) {
                const Inst& I = H.insts[i];
                if (r >= I.nchunks) continue;
                const int sc = std::min(I.S, I.nstrips - r * I.S);
                Segment sg;
                sg.start = t;
                sg.type = ph == 0 ? TASK_TABLE : TASK_GATHER;
                sg.inst = i;
                sg.chunk = r;
                sg.count = ph == 0 ? sc * 2 * I.njb : I.m * 2 * I.njb;
                H.segs.push_back(sg);
                // Segments start at multiples of BLOCK_TASKS: a block's tasks
                // never straddle two segments (padding tasks do nothing).
                t += (sg.count + BLOCK_TASKS - 1) / BLOCK_TASKS * BLOCK_TASKS;
            }
        }
    }
    H.ntasks = t;
    // The queue head is a 32-bit counter that every block bumps by
    // BLOCK_TASKS once past the end.
    if (H.ntasks + (long long)grid * BLOCK_TASKS >= (1LL << 31)) return PCMM_EUNSUPPORTED;
    for (int i = 0; i < count; i++)
        for (int s = 0; s < H.insts[i].nstrips; s++) H.strip_map.push_back(make_int2(i, s));
    H.off_insts = off;   off = align256(off + sizeof(Inst) * count);
    H.off_segs = off;    off = align256(off + sizeof(Segment) * H.segs.size());
    H.off_map = off;     off = align256(off + sizeof(int2) * H.strip_map.size());
    H.off_ctrs = off;    off = align256(off + sizeof(int) * (size_t)H.nctrs);
    H.off_scratch = off; off = align256(off + (size_t)grid * (BATCH_THREADS / 32) * H.scratch_u4 * 16);
    H.bytes = off;
    // Device pointers are filled in by prepare once the workspace is known.
    for (int i = 0; i < count; i++) {
        H.insts[i].A = probs[i].A;
        H.insts[i].ctB = (const uint4*)probs[i].ctB;
        H.insts[i].ctC = (uint4*)probs[i].ctC;
        H.insts[i].P.status = nullptr;
        H.insts[i].tables = (uint4*)(uintptr_t)tab_off[i];   // offset for now
        H.insts[i].P.rank = (uint16_t*)(uintptr_t)plan_off[i];  // offset for now
    }
    // Keep the per-instance Layouts' plan offsets for prepare.
    for (int i = 0; i < count; i++) {
        PlanPtrs P = plan_ptrs(Ls[i], (void*)(uintptr_t)plan_off[i]);
        H.insts[i].P = P;
    }
    return PCMM_OK;
}

int resident_grid() {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel, BATCH_THREADS, 0) !=
        cudaSuccess)
        return 0;
    return sms * std::max(per_sm, 1);
}

}  // namespace

extern "C" size_t pcmm_batched_workspace_bytes(const pcmm_problem* probs, int count, int max_strips) {
    const int grid = resident_grid();
    if (grid <= 0) return 0;
    HostLayout H;
    if (build_layout(probs, count, max_strips, grid, H) != PCMM_OK) return 0;
    return H.bytes;
}

extern "C" pcmm_status pcmm_batched_prepare(const pcmm_problem* probs, int count, int max_strips, void* ws,
                                            size_t ws_bytes, pcmm_batch_info* info, pcmm_stream_t stream) {
    if (!ws || !info || ((uintptr_t)ws & 255u)) return PCMM_EINVAL;
    const int grid = resident_grid();
    if (grid <= 0) return PCMM_ECUDA;
    HostLayout H;
    pcmm_status rc = build_layout(probs, count, max_strips, grid, H);
    if (rc != PCMM_OK) return rc;
    if (ws_bytes < H.bytes) return PCMM_ENOMEM;
    uint8_t* base = (uint8_t*)ws;
    for (auto& I : H.insts) {
        I.tables = (uint4*)(base + (uintptr_t)I.tables);
        PlanPtrs& P = I.P;
        const uintptr_t b = (uintptr_t)base;
        P.rank = (uint16_t*)(b + (uintptr_t)P.rank);
        P.nent = (int32_t*)(b + (uintptr_t)P.nent);
        P.codes = (uint16_t*)(b + (uintptr_t)P.codes);
        P.col_len = (uint16_t*)(b + (uintptr_t)P.col_len);
        P.col_vN = (uint16_t*)(b + (uintptr_t)P.col_vN);
        P.col_ptr = (uint16_t*)(b + (uintptr_t)P.col_ptr);
        P.col_rank1 = (uint8_t*)(b + (uintptr_t)P.col_rank1);
        P.status = (uint32_t*)base;        // all instances report into the batch status word
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(base + H.off_insts, H.insts.data(), sizeof(Inst) * H.insts.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(base + H.off_segs, H.segs.data(), sizeof(Segment) * H.segs.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(base + H.off_map, H.strip_map.data(), sizeof(int2) * H.strip_map.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return PCMM_ECUDA;
    // The host vectors die on return: wait for the copies.
    if (cudaStreamSynchronize(st) != cudaSuccess) return PCMM_ECUDA;
    info->count = count;
    info->nsegs = (int)H.segs.size();
    info->ntasks = H.ntasks;
    info->nstrips = (long long)H.strip_map.size();
    info->nctrs = H.nctrs;
    info->grid = H.grid;
    info->off_insts = H.off_insts;
    info->off_segs = H.off_segs;
    info->off_map = H.off_map;
    info->off_ctrs = H.off_ctrs;
    info->off_scratch = H.off_scratch;
    info->scratch_u4 = H.scratch_u4;
    info->bytes = H.bytes;
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_batched_run(const pcmm_batch_info* info, void* ws, pcmm_stream_t stream) {
    if (!info || !ws || ((uintptr_t)ws & 255u) || info->grid < 1 || info->nstrips < 1) return PCMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    uint8_t* base = (uint8_t*)ws;
    if (cudaMemsetAsync(base, 0, sizeof(BatchHeader), st) != cudaSuccess ||
        cudaMemsetAsync(base + info->off_ctrs, 0, sizeof(int) * (size_t)info->nctrs, st) != cudaSuccess)
        return PCMM_ECUDA;
    const Inst* insts = (const Inst*)(base + info->off_insts);
    {
        ProfScope ps(KID_PLAN, st);
        batched_plan_kernel<<<(unsigned)info->nstrips, PLAN_THREADS, 0, st>>>(
            insts, (const int2*)(base + info->off_map));
    }
    PCMM_CUDA_CHECK_LAUNCH();
    {
        ProfScope ps(KID_BATCHED, st);
        batched_kernel<<<(unsigned)info->grid, BATCH_THREADS, 0, st>>>(
            insts, (const Segment*)(base + info->off_segs), info->nsegs, info->ntasks, (BatchHeader*)base,
            (int*)(base + info->off_ctrs), (uint4*)(base + info->off_scratch), info->scratch_u4);
    }
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_cussen_batched(const pcmm_problem* probs, int count, void* ws, size_t ws_bytes,
                                           pcmm_stream_t stream) {
    if (!probs || count < 1 || !ws) return PCMM_EINVAL;
    pcmm_batch_info info;
    const pcmm_status rc = pcmm_batched_prepare(probs, count, 0, ws, ws_bytes, &info, stream);
    if (rc != PCMM_OK) return rc;
    return pcmm_batched_run(&info, ws, stream);
}
