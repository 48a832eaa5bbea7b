// Optional per-kernel timing with CUDA events recorded on the launching
// stream around every library kernel launch (off by default).
#pragma once
#include <cuda_runtime.h>

namespace pcmm {

enum KernelId {
    KID_PLAN = 0,
    KID_TABLE = 1,
    KID_GATHER = 2,
    KID_NORMALIZE = 3,
    KID_ENCRYPT = 4,
    KID_SCHOOLBOOK = 5,
    KID_COMB = 6,
    KID_BATCHED = 7,
    KID_COMBINE = 8,
    KID_BSGS = 9,
    KID_DECRYPT = 10,
    KID_STRASSEN_SUM = 11,
    KID_STRASSEN_LEAF = 12,
    KID_STRASSEN_COMBINE = 13,
    KID_COUNT = 14
};

// Records a start event on construction and a stop event on destruction
// when profiling is enabled; otherwise does nothing.
struct ProfScope {
    int slot;
    cudaStream_t stream;
    ProfScope(int kernel_id, cudaStream_t s);
    ~ProfScope();
};

}  // namespace pcmm
