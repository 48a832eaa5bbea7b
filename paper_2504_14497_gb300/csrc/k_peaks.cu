// Integer-pipe throughput microbenchmark: the measured denominators of the
// roofline that bounds the PC-MM kernels (exact modular arithmetic runs on
// the integer multiply-add and ALU pipes, not on tensor cores).
//
// Every thread runs eight independent chains of one instruction kind in
// inline PTX, each instruction depending on the previous one of its chain so
// that nothing can be folded or hoisted out of the loop, for `iters`
// iterations; the chains' final values are XOR-ed into one word of `sink` so
// that no chain is dead code.  A grid of whole waves over all SMs keeps every
// scheduler busy; ops per second = threads x iters x ops per iteration /
// kernel time.
#include <cuda_runtime.h>

#include "../../include/pcmm.h"
#include "common.cuh"

namespace {

constexpr int PEAK_THREADS = 256;

__global__ void __launch_bounds__(PEAK_THREADS) peak_kernel(int op, int iters, uint32_t* __restrict__ sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[8], b = t * 2654435761u + 1u, c = t ^ 0x9e3779b9u;
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = t + 977u * (uint32_t)i;
    uint64_t d[8];
#pragma unroll
    for (int i = 0; i < 8; i++) d[i] = ((uint64_t)a[i] << 17) ^ c;
    if (op == PCMM_PEAK_MAD_LO) {
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 8; i++) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
        }
    } else if (op == PCMM_PEAK_MAD_HI) {
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 8; i++) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(b), "r"(c));
        }
    } else if (op == PCMM_PEAK_MAD_WIDE) {
        for (int it = 0; it < iters; it++) {
#pragma unroll
            // Chains 2q and 2q + 1 feed each other: each product's
            // multiplicand is the low word of the other chain's latest
            // value (a fixed multiplicand would let the assembler hoist the
            // product; one taken from the accumulator's own register pair
            // measured at a third of the rate).
            for (int i = 0; i < 8; i++)
                asm volatile("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %1;\n\t"
                             "mad.wide.u32 %0, lo, %2, %0;\n\t}" : "+l"(d[i]) : "l"(d[i ^ 1]), "r"(b));
        }
    } else if (op == PCMM_PEAK_MUL_WIDE) {
        // Each product's multiplicand is the low word of its chain's
        // previous product: one 32 x 32 -> 64-bit product per instruction.
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 8; i++)
                asm volatile("{\n\t.reg .b32 lo, hi;\n\tmov.b64 {lo, hi}, %0;\n\t"
                             "mul.wide.u32 %0, lo, %1;\n\t}" : "+l"(d[i]) : "r"(b));
        }
    } else if (op == PCMM_PEAK_ADD_CARRY) {
        // Two independent 4-limb additions with carry per iteration:
        // add.cc, addc.cc, addc.cc, addc (the carry chains of multi-limb
        // field arithmetic).
        for (int it = 0; it < iters; it++) {
            asm volatile(
                "add.cc.u32 %0, %0, %8;\n\t"
                "addc.cc.u32 %1, %1, %9;\n\t"
                "addc.cc.u32 %2, %2, %8;\n\t"
                "addc.u32 %3, %3, %9;\n\t"
                "add.cc.u32 %4, %4, %9;\n\t"
                "addc.cc.u32 %5, %5, %8;\n\t"
                "addc.cc.u32 %6, %6, %9;\n\t"
                "addc.u32 %7, %7, %8;"
                : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]),
                  "+r"(a[7])
                : "r"(b), "r"(c));
        }
    } else {  // PCMM_PEAK_ADD
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 8; i++) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) x ^= a[i] ^ (uint32_t)d[i] ^ (uint32_t)(d[i] >> 32);
    if (x == 0x5eed5eedu) sink[t & 1023u] = x;   // practically never taken; keeps the chains live
}

}  // namespace

extern "C" int pcmm_peak_ops_per_iter(int op) {
    return (op >= PCMM_PEAK_MAD_LO && op <= PCMM_PEAK_MUL_WIDE) ? 8 : 0;
}

extern "C" int pcmm_peak_threads_per_block(void) { return PEAK_THREADS; }

extern "C" pcmm_status pcmm_peak_run(int op, int blocks, int iters, uint32_t* sink, pcmm_stream_t stream) {
    if (!pcmm_peak_ops_per_iter(op) || blocks < 1 || iters < 1 || !sink) return PCMM_EINVAL;
    peak_kernel<<<(unsigned)blocks, PEAK_THREADS, 0, (cudaStream_t)stream>>>(op, iters, sink);
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}
