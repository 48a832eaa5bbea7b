// Cussen PC-MM for callers that cannot allocate device memory.
//
// Some callers are only handed their input and output buffers and may not
// call cudaMalloc: a plug-in inside a host framework that owns the whole
// device memory pool, a latency-critical loop that cannot afford the
// implicit synchronisation and unpredictable latency of an allocation, or a
// process whose memory cap is already fully reserved.  pcmm_cussen_static
// gives them the same computation as pcmm_cussen, with the scratch space
// taken from a fixed array that the library itself reserves in global memory.
#include <atomic>

#include <cuda_runtime.h>

#include "../../include/pcmm.h"

namespace {

// 32 MiB: enough for the 1024 x 1024 x 256 problem at w = 8 (its plan plus
// one strip is 31.2 MB).  Every GPU on which the library is loaded holds this
// array until the process exits.
constexpr size_t STATIC_SCRATCH_BYTES = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_scratch[STATIC_SCRATCH_BYTES];

// Device address of g_scratch for each device, looked up once per device with
// that device current.  In host code the name g_scratch is only a host-side
// stand-in for the symbol, never a usable device pointer.  Concurrent first
// calls from several host threads may each look it up; they store the same
// value.
constexpr int MAX_DEVICES = 64;
std::atomic<void*> g_scratch_addr[MAX_DEVICES];

}  // namespace

extern "C" pcmm_status pcmm_cussen_static(const uint8_t* A, int m, int n, int w, const uint32_t* ctB,
                                          int l, uint32_t* ctC, int k, uint32_t* status,
                                          pcmm_stream_t stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PCMM_ECUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return PCMM_EUNSUPPORTED;
    void* scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!scratch) {
        if (cudaGetSymbolAddress(&scratch, g_scratch) != cudaSuccess || !scratch) return PCMM_ECUDA;
        g_scratch_addr[dev].store(scratch, std::memory_order_release);
    }
    // pcmm_cussen clears the status word at the start of the scratch; every
    // other byte it reads in a call is written earlier in that call.
    const pcmm_status st = pcmm_cussen(A, m, n, w, ctB, l, ctC, k, scratch, STATIC_SCRATCH_BYTES, stream);
    if (st != PCMM_OK) return st == PCMM_ENOMEM ? PCMM_EUNSUPPORTED : st;
    // The kernels' error bits live in the private scratch: hand them over.
    if (status && cudaMemcpyAsync(status, scratch, 4, cudaMemcpyDefault, (cudaStream_t)stream) != cudaSuccess)
        return PCMM_ECUDA;
    return PCMM_OK;
}
