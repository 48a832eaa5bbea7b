// Per-kernel CUDA-event timing (see profiler.cuh).  A fixed pool of event
// pairs is created by pcmm_profile_enable; each profiled launch takes the
// next pair.  Not thread-safe: enable, run and read from one host thread.
// Every launch is also wrapped in an NVTX range named after its kernel (a
// no-op unless a tracing tool is attached).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "../../include/pcmm.h"
#include "profiler.cuh"

namespace pcmm {
namespace {
struct Slot {
    cudaEvent_t start, stop;
    int kid;
};
std::vector<Slot> g_slots;
int g_used = 0;
bool g_on = false;
const char* const g_names[KID_COUNT] = {"plan", "table", "gather", "normalize",
                                        "encrypt", "schoolbook", "comb", "batched", "combine",
                                        "bsgs", "decrypt", "strassen_sum", "strassen_leaf",
                                        "strassen_combine"};
}  // namespace

ProfScope::ProfScope(int kernel_id, cudaStream_t s) : slot(-1), stream(s) {
    nvtxRangePushA(kernel_id >= 0 && kernel_id < KID_COUNT ? g_names[kernel_id] : "pcmm");
    if (!g_on || g_used >= (int)g_slots.size()) return;
    slot = g_used++;
    g_slots[slot].kid = kernel_id;
    cudaEventRecord(g_slots[slot].start, s);
}

ProfScope::~ProfScope() {
    if (slot >= 0) cudaEventRecord(g_slots[slot].stop, stream);
    nvtxRangePop();
}

}  // namespace pcmm

using namespace pcmm;

extern "C" pcmm_status pcmm_profile_enable(int capacity) {
    for (auto& s : g_slots) {
        cudaEventDestroy(s.start);
        cudaEventDestroy(s.stop);
    }
    g_slots.clear();
    g_used = 0;
    g_on = false;
    if (capacity <= 0) return PCMM_OK;
    g_slots.resize((size_t)capacity);
    for (auto& s : g_slots) {
        if (cudaEventCreate(&s.start) != cudaSuccess || cudaEventCreate(&s.stop) != cudaSuccess)
            return PCMM_ECUDA;
        s.kid = -1;
    }
    g_on = true;
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_profile_read(double* ms, long long* launches) {
    if (!ms || !launches) return PCMM_EINVAL;
    for (int k = 0; k < KID_COUNT; k++) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (int i = 0; i < g_used; i++) {
        float t = 0.f;
        if (cudaEventSynchronize(g_slots[i].stop) != cudaSuccess) return PCMM_ECUDA;
        if (cudaEventElapsedTime(&t, g_slots[i].start, g_slots[i].stop) != cudaSuccess) return PCMM_ECUDA;
        ms[g_slots[i].kid] += t;
        launches[g_slots[i].kid] += 1;
    }
    g_used = 0;
    return PCMM_OK;
}

extern "C" const char* pcmm_kernel_name(int id) {
    return (id >= 0 && id < KID_COUNT) ? g_names[id] : "unknown";
}

extern "C" int pcmm_kernel_count(void) { return KID_COUNT; }
