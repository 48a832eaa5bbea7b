// Schoolbook PC-MM (Section 3.1): Enc(c_ij) = sum_k a_ik Enc(b_kj), each
// plaintext-ciphertext product by double-and-add, accumulated by point
// additions.  The in-library baseline for Cussen's method.
//
// Mapping: one warp per (row i, component c, block of 32 output columns);
// lane L handles column j = 32 * block + L.  a_ik is the same for the whole
// warp, so the double-and-add control flow is warp-uniform, and the lanes'
// loads of B_c^(kj) for consecutive j are coalesced.
#include <cuda_runtime.h>

#include "common.cuh"
#include "profiler.cuh"

using namespace pcmm;

namespace {

template <class TA>
__global__ void __launch_bounds__(128) schoolbook_kernel(const TA* __restrict__ A, int m,
                                                         int n, const uint4* __restrict__ ctB,
                                                         int l, uint4* __restrict__ ctC,
                                                         uint32_t amask) {
    const unsigned lane = threadIdx.x & 31u;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nJB = (l + 31) / 32;
    const long long total = (long long)m * 2 * nJB;
    if (gw >= total) return;
    const int i = (int)(gw / (2 * nJB));
    const int rem = (int)(gw % (2 * nJB));
    const int c = rem / nJB, jb = rem % nJB;
    const int j = jb * 32 + (int)lane;
    const int jj = j < l ? j : l - 1;
    const size_t nl = (size_t)n * l, ml = (size_t)m * l;
    const uint4* Bc = ctB + (size_t)c * 4 * nl;
    jac acc, term;
    jac_set_inf(acc);
    aff P;
    for (int k = 0; k < n; k++) {
        const uint32_t a = A[(size_t)i * n + k] & amask;
        if (a == 0u) continue;
        load_aff(P, Bc, nl, (size_t)k * l + jj);
        jac_mul_small(term, P, a);
        jac_add(acc, term);
    }
    if (j < l) store_jac(ctC + (size_t)c * 6 * ml, ml, (size_t)i * l + j, acc);
}

template <class TA>
pcmm_status schoolbook_call(const TA* A, int m, int n, int w, const uint32_t* ctB, int l, uint32_t* ctC,
                            pcmm_stream_t stream) {
    if (!A || !ctB || !ctC || m < 1 || n < 1 || l < 1 || w < 1 || w > 8 * (int)sizeof(TA))
        return PCMM_EINVAL;
    const long long warps = (long long)m * 2 * ((l + 31) / 32);
    const long long blocks = (warps + 3) / 4;
    if (blocks > 0x7fffffffLL) return PCMM_EUNSUPPORTED;
    ProfScope ps(KID_SCHOOLBOOK, (cudaStream_t)stream);
    schoolbook_kernel<TA><<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(
        A, m, n, (const uint4*)ctB, l, (uint4*)ctC, (1u << w) - 1u);
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

}  // namespace

extern "C" pcmm_status pcmm_schoolbook(const uint8_t* A, int m, int n, int w, const uint32_t* ctB,
                                       int l, uint32_t* ctC, pcmm_stream_t stream) {
    return schoolbook_call(A, m, n, w, ctB, l, ctC, stream);
}

extern "C" pcmm_status pcmm_schoolbook16(const uint16_t* A, int m, int n, int w, const uint32_t* ctB,
                                         int l, uint32_t* ctC, pcmm_stream_t stream) {
    return schoolbook_call(A, m, n, w, ctB, l, ctC, stream);
}
