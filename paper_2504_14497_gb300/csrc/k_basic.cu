// Encryption (Section 2.4), output normalisation, and unit-test entry points
// for the device field and group arithmetic.
#include <cuda_runtime.h>

#include "comb.cuh"
#include "common.cuh"
#include "profiler.cuh"

using namespace pcmm;

namespace {

// Comb table of the generator, quad-planar with stride COMB_POINTS.
__device__ uint4 g_comb_G[4 * COMB_POINTS];

// P-256 generator (SEC 2 / FIPS 186-4), little-endian 32-bit words.
const uint32_t h_G[16] = {
    0xd898c296u, 0xf4a13945u, 0x2deb33a0u, 0x77037d81u, 0x63a440f2u, 0xf8bce6e5u, 0xe12c4247u, 0x6b17d1f2u,
    0x37bf51f5u, 0xcbb64068u, 0x6b315eceu, 0x2bce3357u, 0x7c0f9e16u, 0x8ee7eb4au, 0xfe1a7f9bu, 0x4fe342e2u};

// R <- s P for a 256-bit scalar s (8 little-endian words) by left-to-right
// double-and-add with mixed additions of the affine P.
__device__ void jac_mul_u256(jac& R, const aff& P, const uint32_t s[8]) {
    jac_set_inf(R);
    bool started = false;
    for (int b = 255; b >= 0; b--) {
        if (started) jac_dbl(R);
        if ((s[b >> 5] >> (b & 31)) & 1u) {
            jac_madd(R, P);
            started = true;
        }
    }
}

// Entry (window i, value v) = (v 2^(8i)) X.  One thread per entry; the
// results are normalised one warp at a time.
__global__ void __launch_bounds__(128) comb_build_kernel(aff base, uint4* __restrict__ tab) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // < COMB_POINTS
    const int win = idx / COMB_ENTRIES, v = idx % COMB_ENTRIES;
    uint32_t s[8];
#pragma unroll
    for (int i = 0; i < 8; i++) s[i] = 0;
    s[win >> 2] = (uint32_t)v << (8 * (win & 3));
    jac R[1];
    jac_mul_u256(R[0], base, s);
    aff out[1];
    warp_normalize_regs<1>(out, R);
    store_aff(tab, COMB_POINTS, idx, out[0]);
}

// Header of an encryption workspace: a tag word, then the 16 words of the
// point whose comb table follows.  The build below skips its work when the
// header already names the requested point.
constexpr uint32_t KEY_TAG = 0x4b455931u;
constexpr size_t ENC_HDR_BYTES = 256;

__device__ __forceinline__ bool header_names(const uint32_t* __restrict__ hdr, const aff& X) {
    bool same = hdr[0] == KEY_TAG;
#pragma unroll
    for (int i = 0; i < 8; i++) same &= (hdr[1 + i] == X.x.v[i]) & (hdr[9 + i] == X.y.v[i]);
    return same;
}

// comb_build_kernel unless the header already names `base`.  Every block
// reads the header before the tag kernel (next in stream order) writes it.
__global__ void __launch_bounds__(128) comb_build_cached_kernel(aff base, const uint32_t* __restrict__ hdr,
                                                                uint4* __restrict__ tab) {
    if (header_names(hdr, base)) return;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int win = idx / COMB_ENTRIES, v = idx % COMB_ENTRIES;
    uint32_t s[8];
#pragma unroll
    for (int i = 0; i < 8; i++) s[i] = 0;
    s[win >> 2] = (uint32_t)v << (8 * (win & 3));
    jac R[1];
    jac_mul_u256(R[0], base, s);
    aff out[1];
    warp_normalize_regs<1>(out, R);
    store_aff(tab, COMB_POINTS, idx, out[0]);
}

// Clears the tag when the header names another point, so that a table left
// half rebuilt by a call that failed after this point is never reused.
__global__ void comb_untag_kernel(aff base, uint32_t* __restrict__ hdr) {
    if (threadIdx.x == 0 && !header_names(hdr, base)) hdr[0] = 0;
}

__global__ void comb_tag_kernel(aff base, uint32_t* __restrict__ hdr) {
    const int i = threadIdx.x;
    if (i < 8) {
        hdr[1 + i] = base.x.v[i];
        hdr[9 + i] = base.y.v[i];
    }
    if (i == 0) hdr[0] = KEY_TAG;
}

// Enc(b) = (rG, rH + bG): 32 window lookups per base point.
__global__ void __launch_bounds__(128) encrypt_kernel(const uint4* __restrict__ gtab,
                                                      const uint4* __restrict__ htab,
                                                      const uint8_t* __restrict__ msg,
                                                      const uint4* __restrict__ r, size_t count,
                                                      uint4* __restrict__ ct) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < count;
    const size_t ii = valid ? i : 0;
    fe rr;
    fe_from_quads(rr, r[ii], r[count + ii]);
    jac P[2];
    jac_set_inf(P[0]);
    jac_set_inf(P[1]);
    aff T;
    for (int win = 0; win < COMB_WINDOWS; win++) {
        const uint32_t v = (rr.v[win >> 2] >> (8 * (win & 3))) & 0xffu;
        if (v) {
            load_aff(T, gtab, COMB_POINTS, (size_t)win * COMB_ENTRIES + v);
            jac_madd(P[0], T);
            load_aff(T, htab, COMB_POINTS, (size_t)win * COMB_ENTRIES + v);
            jac_madd(P[1], T);
        }
    }
    const uint32_t b = msg[ii];
    if (b) {
        load_aff(T, gtab, COMB_POINTS, b);
        jac_madd(P[1], T);
    }
    aff out[2];
    warp_normalize_regs<2>(out, P);
    if (valid) {
        store_aff(ct, count, i, out[0]);
        store_aff(ct + 4 * count, count, i, out[1]);
    }
}

// s G for count scalars (key generation: H = x G), one thread per scalar.
__global__ void __launch_bounds__(128) base_mul_kernel(const uint4* __restrict__ gtab,
                                                       const uint4* __restrict__ sc, size_t count,
                                                       uint4* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < count;
    const size_t ii = valid ? i : 0;
    fe s;
    fe_from_quads(s, sc[ii], sc[count + ii]);
    jac P[1];
    jac_set_inf(P[0]);
    aff T;
    for (int win = 0; win < COMB_WINDOWS; win++) {
        const uint32_t v = (s.v[win >> 2] >> (8 * (win & 3))) & 0xffu;
        if (v) {
            load_aff(T, gtab, COMB_POINTS, (size_t)win * COMB_ENTRIES + v);
            jac_madd(P[0], T);
        }
    }
    aff o[1];
    warp_normalize_regs<1>(o, P);
    if (valid) store_aff(out, count, i, o[0]);
}

// Jacobian ciphertexts -> canonical affine.  Thread t takes the G
// ciphertexts i = g T + t (T threads in the grid, g < G; each g is a
// coalesced sweep), that is 2G points, and the block's 128 threads share
// one field inversion among their 256 G points (Montgomery's simultaneous
// inversion: prefix products across each lane's points, across the warp by
// shuffles, across the block's four warps).
// The prefix products wait in the output's x words, which the
// backward pass overwrites point by point after reading them.
__global__ void __launch_bounds__(128) normalize_kernel(const uint4* __restrict__ in, size_t count,
                                                        uint4* __restrict__ out, int G) {
    const unsigned lane = threadIdx.x & 31u;
    const size_t T = (size_t)gridDim.x * blockDim.x;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    fe acc;
    fe_one(acc);
    bool ones = true;
    for (int g = 0; g < G; g++) {
        const size_t i = (size_t)g * T + t;
        if (i >= count) break;
#pragma unroll
        for (int c = 0; c < 2; c++) {
            const uint4* b = in + (size_t)c * 6 * count;
            fe z;
            fe_from_quads(z, b[4 * count + i], b[5 * count + i]);
            ones &= fe_is_one(z);
            if (fe_is_zero(z)) fe_one(z);
            acc = fmul(acc, z);
            uint4* o = out + (size_t)c * 4 * count;
            o[i] = fe_lo(acc);
            o[count + i] = fe_hi(acc);
        }
    }
    // Every thread of the (128-thread) block reaches this point, with or
    // without ciphertexts, so the block votes and shares one inversion.
    if (group_all(ones, true)) {
        for (int g = 0; g < G; g++) {
            const size_t i = (size_t)g * T + t;
            if (i >= count) break;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                jac P;
                load_jac(P, in + (size_t)c * 6 * count, count, i);
                aff A;
                fe_canon(A.x, P.X);
                fe_canon(A.y, P.Y);
                store_aff(out + (size_t)c * 4 * count, count, i, A);
            }
        }
        return;
    }
    fe inv;
    group_inverse(inv, acc, true);
    for (int g = G - 1; g >= 0; g--) {
        const size_t i = (size_t)g * T + t;
        if (i >= count) continue;
#pragma unroll
        for (int c = 1; c >= 0; c--) {
            // The point before (g, c) in the forward order holds the prefix.
            fe zinv;
            if (c == 1 || g > 0) {
                const size_t ip = c == 1 ? i : i - T;
                const uint4* o = out + (size_t)(c == 1 ? 0 : 1) * 4 * count;
                fe pr;
                fe_from_quads(pr, o[ip], o[count + ip]);
                zinv = fmul(inv, pr);
            } else {
                zinv = inv;
            }
            jac P;
            load_jac(P, in + (size_t)c * 6 * count, count, i);
            fe z = P.Z;
            const bool is_inf = fe_is_zero(z);
            if (is_inf) fe_one(z);
            inv = fmul(inv, z);
            aff A;
            if (is_inf) {
                fe_zero(A.x);
                fe_zero(A.y);
            } else {
                jac_to_aff_with_zinv(A, P, zinv);
            }
            store_aff(out + (size_t)c * 4 * count, count, i, A);
        }
    }
}

__global__ void __launch_bounds__(128) test_field_kernel(int op, const uint4* __restrict__ a,
                                                         const uint4* __restrict__ b,
                                                         uint4* __restrict__ out, size_t count) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    fe x, y, r;
    load_fe(x, a, count, i);
    if (op <= 2) load_fe(y, b, count, i);
    switch (op) {
        case 0: fe_add(r, x, y); break;
        case 1: fe_sub(r, x, y); break;
        case 2: fe_mul(r, x, y); break;
        case 3: fe_sqr(r, x); break;
        case 4: fe_inv(r, x); break;
        default: r = x; break;
    }
    fe_canon(r, r);
    store_fe(out, count, i, r);
}

__global__ void __launch_bounds__(128) test_point_kernel(int op, const uint4* __restrict__ P,
                                                         const uint4* __restrict__ Q,
                                                         const uint32_t* __restrict__ ks,
                                                         uint4* __restrict__ out, size_t count) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < count;
    const size_t ii = valid ? i : 0;
    jac R[1];
    if (op == 3) {
        aff A;
        load_aff(A, P, count, ii);
        jac_mul_small(R[0], A, ks[ii]);
    } else {
        load_jac(R[0], P, count, ii);
        if (op == 0) {
            jac_dbl(R[0]);
        } else if (op == 1) {
            aff B;
            load_aff(B, Q, count, ii);
            jac_madd(R[0], B);
        } else {
            jac B;
            load_jac(B, Q, count, ii);
            jac_add(R[0], B);
        }
    }
    aff o[1];
    warp_normalize_regs<1>(o, R);
    if (valid) store_aff(out, count, i, o[0]);
}

// Every warp waits (bounded) for *ctr >= target; lane 0 records in out[warp]
// whether the target was reached.
__global__ void test_wait_kernel(const int* ctr, int target, uint32_t* status, int* out) {
    if ((threadIdx.x & 31u) == 0) {
        const bool ok = wait_at_least(ctr, target, status);
        out[(blockIdx.x * blockDim.x + threadIdx.x) >> 5] = ok ? 1 : 0;
    }
}

inline unsigned grid_for(size_t count, unsigned block) { return (unsigned)((count + block - 1) / block); }

bool g_ready[64] = {false};

}  // namespace

const uint4* pcmm::comb_table_G() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || !g_ready[dev]) return nullptr;
    uint4* tab = nullptr;
    if (cudaGetSymbolAddress((void**)&tab, g_comb_G) != cudaSuccess) return nullptr;
    return tab;
}

extern "C" int pcmm_version(void) { return 10000; }

extern "C" const char* pcmm_status_string(int s) {
    switch (s) {
        case PCMM_OK: return "PCMM_OK";
        case PCMM_EINVAL: return "PCMM_EINVAL: invalid argument";
        case PCMM_ENOMEM: return "PCMM_ENOMEM: workspace too small";
        case PCMM_ECUDA: return "PCMM_ECUDA: CUDA error";
        case PCMM_ETIMEOUT: return "PCMM_ETIMEOUT: device wait timed out";
        case PCMM_EUNSUPPORTED: return "PCMM_EUNSUPPORTED: unsupported request";
        case PCMM_EDEVICE: return "PCMM_EDEVICE: a kernel flagged invalid data";
        default: return "unknown pcmm status";
    }
}

extern "C" pcmm_status pcmm_init(int device) {
    if (device < 0 || device >= 64) return PCMM_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) return PCMM_ECUDA;
    if (g_ready[device]) return PCMM_OK;
    aff G;
    for (int i = 0; i < 8; i++) {
        G.x.v[i] = h_G[i];
        G.y.v[i] = h_G[8 + i];
    }
    uint4* tab = nullptr;
    if (cudaGetSymbolAddress((void**)&tab, g_comb_G) != cudaSuccess) return PCMM_ECUDA;
    {
        ProfScope ps(KID_COMB, 0);
        comb_build_kernel<<<COMB_POINTS / 128, 128>>>(G, tab);
    }
    PCMM_CUDA_CHECK_LAUNCH();
    if (cudaDeviceSynchronize() != cudaSuccess) return PCMM_ECUDA;
    g_ready[device] = true;
    return PCMM_OK;
}

extern "C" size_t pcmm_keytable_bytes(void) { return (size_t)COMB_POINTS * 64; }

static bool reduced_below_p(const uint32_t* v) {
    static const uint32_t p[8] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 1u, 0xffffffffu};
    for (int i = 7; i >= 0; i--) {
        if (v[i] < p[i]) return true;
        if (v[i] > p[i]) return false;
    }
    return false;
}

// Validates a host public key and copies it into an affine point.
static pcmm_status key_from_host(const uint32_t* H_host, aff& H) {
    if (!H_host) return PCMM_EINVAL;
    if (!reduced_below_p(H_host) || !reduced_below_p(H_host + 8)) return PCMM_EINVAL;
    uint32_t z = 0;
    for (int i = 0; i < 8; i++) {
        H.x.v[i] = H_host[i];
        H.y.v[i] = H_host[8 + i];
        z |= H_host[i] | H_host[8 + i];
    }
    return z ? PCMM_OK : PCMM_EINVAL;
}

extern "C" pcmm_status pcmm_keytable(const uint32_t* H_host, void* keytable, pcmm_stream_t stream) {
    aff H;
    if (!keytable || ((uintptr_t)keytable & 15u) || key_from_host(H_host, H) != PCMM_OK) return PCMM_EINVAL;
    {
        ProfScope ps(KID_COMB, (cudaStream_t)stream);
        comb_build_kernel<<<COMB_POINTS / 128, 128, 0, (cudaStream_t)stream>>>(H, (uint4*)keytable);
    }
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

static pcmm_status launch_encrypt(const void* keytable, const uint8_t* msg, const uint32_t* r, size_t count,
                                  uint32_t* ct, cudaStream_t st) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PCMM_ECUDA;
    if (dev < 0 || dev >= 64 || !g_ready[dev]) return PCMM_EINVAL;
    uint4* gtab = nullptr;
    if (cudaGetSymbolAddress((void**)&gtab, g_comb_G) != cudaSuccess) return PCMM_ECUDA;
    ProfScope ps(KID_ENCRYPT, st);
    encrypt_kernel<<<grid_for(count, 128), 128, 0, st>>>(gtab, (const uint4*)keytable, msg, (const uint4*)r,
                                                         count, (uint4*)ct);
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_encrypt_table(const void* keytable, const uint8_t* msg, const uint32_t* r,
                                          size_t count, uint32_t* ct, pcmm_stream_t stream) {
    if (!keytable || !msg || !r || !ct) return PCMM_EINVAL;
    if (count == 0) return PCMM_OK;
    return launch_encrypt(keytable, msg, r, count, ct, (cudaStream_t)stream);
}

extern "C" size_t pcmm_encrypt_workspace_bytes(void) { return ENC_HDR_BYTES + (size_t)COMB_POINTS * 64; }

extern "C" pcmm_status pcmm_encrypt(const uint32_t* H_host, const uint8_t* msg, const uint32_t* r, size_t count,
                                    uint32_t* ct, void* ws, size_t ws_bytes, pcmm_stream_t stream) {
    aff H;
    if (key_from_host(H_host, H) != PCMM_OK) return PCMM_EINVAL;
    if ((count && (!msg || !r || !ct)) || !ws || ((uintptr_t)ws & 255u)) return PCMM_EINVAL;
    if (ws_bytes < pcmm_encrypt_workspace_bytes()) return PCMM_ENOMEM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PCMM_ECUDA;
    if (dev < 0 || dev >= 64 || !g_ready[dev]) return PCMM_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* hdr = (uint32_t*)ws;
    uint4* tab = (uint4*)((uint8_t*)ws + ENC_HDR_BYTES);
    comb_untag_kernel<<<1, 32, 0, st>>>(H, hdr);
    PCMM_CUDA_CHECK_LAUNCH();
    {
        ProfScope ps(KID_COMB, st);
        comb_build_cached_kernel<<<COMB_POINTS / 128, 128, 0, st>>>(H, hdr, tab);
    }
    PCMM_CUDA_CHECK_LAUNCH();
    comb_tag_kernel<<<1, 32, 0, st>>>(H, hdr);
    PCMM_CUDA_CHECK_LAUNCH();
    if (count == 0) return PCMM_OK;
    return launch_encrypt(tab, msg, r, count, ct, st);
}

extern "C" pcmm_status pcmm_base_mul(const uint32_t* scalars, size_t count, uint32_t* points,
                                     pcmm_stream_t stream) {
    if (!scalars || !points) return PCMM_EINVAL;
    if (count == 0) return PCMM_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PCMM_ECUDA;
    if (dev < 0 || dev >= 64 || !g_ready[dev]) return PCMM_EINVAL;
    uint4* gtab = nullptr;
    if (cudaGetSymbolAddress((void**)&gtab, g_comb_G) != cudaSuccess) return PCMM_ECUDA;
    ProfScope ps(KID_ENCRYPT, (cudaStream_t)stream);
    base_mul_kernel<<<grid_for(count, 128), 128, 0, (cudaStream_t)stream>>>(
        gtab, (const uint4*)scalars, count, (uint4*)points);
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_normalize(const uint32_t* ct_jac, size_t count, uint32_t* ct_aff,
                                      pcmm_stream_t stream) {
    if (!ct_jac || !ct_aff) return PCMM_EINVAL;
    if (count == 0) return PCMM_OK;
    ProfScope ps(KID_NORMALIZE, (cudaStream_t)stream);
#ifdef PCMM_NORM_G
    const int G = PCMM_NORM_G;
#else
    // G ciphertexts per thread while at least NORM_MIN_THREADS threads remain:
    // measured on 262144 ciphertexts (four per headline step), 3.50 ms per
    // step at G = 1, 1.92 at 2, 1.30 at 4, 0.90 at 8.
    const size_t NORM_MIN_THREADS = 32768;
    int G = 1;
    while (G < 8 && count / (size_t)(2 * G) >= NORM_MIN_THREADS) G *= 2;
#endif
    const size_t threads = (count + G - 1) / G;
    normalize_kernel<<<grid_for(threads, 128), 128, 0, (cudaStream_t)stream>>>(
        (const uint4*)ct_jac, count, (uint4*)ct_aff, G);
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_copy_columns(uint32_t* dst, size_t dst_ld, size_t dst_col,
                                         const uint32_t* src, size_t src_ld, size_t src_col,
                                         size_t ncols, size_t nrows, pcmm_stream_t stream) {
    if (!dst || !src || ncols > dst_ld || ncols > src_ld || dst_col + ncols > dst_ld ||
        src_col + ncols > src_ld)
        return PCMM_EINVAL;
    if (ncols == 0 || nrows == 0) return PCMM_OK;
    if (cudaMemcpy2DAsync((uint8_t*)dst + dst_col * 16, dst_ld * 16, (const uint8_t*)src + src_col * 16,
                          src_ld * 16, ncols * 16, nrows, cudaMemcpyDefault,
                          (cudaStream_t)stream) != cudaSuccess)
        return PCMM_ECUDA;
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_test_wait(const int* ctr, int target, uint32_t* status, int* out, int warps,
                                      pcmm_stream_t stream) {
    if (!ctr || !status || !out || warps < 1 || warps > 1024) return PCMM_EINVAL;
    test_wait_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, (cudaStream_t)stream>>>(ctr, target, status, out);
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_test_field(int op, const uint32_t* a, const uint32_t* b, uint32_t* out,
                                       size_t count, pcmm_stream_t stream) {
    if (op < 0 || op > 5 || !a || !out || (op <= 2 && !b)) return PCMM_EINVAL;
    if (count == 0) return PCMM_OK;
    test_field_kernel<<<grid_for(count, 128), 128, 0, (cudaStream_t)stream>>>(
        op, (const uint4*)a, (const uint4*)b, (uint4*)out, count);
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}

extern "C" pcmm_status pcmm_test_point(int op, const uint32_t* P, const uint32_t* Q,
                                       const uint32_t* kscal, uint32_t* out, size_t count,
                                       pcmm_stream_t stream) {
    if (op < 0 || op > 3 || !P || !out || ((op == 1 || op == 2) && !Q) || (op == 3 && !kscal))
        return PCMM_EINVAL;
    if (count == 0) return PCMM_OK;
    test_point_kernel<<<grid_for(count, 128), 128, 0, (cudaStream_t)stream>>>(
        op, (const uint4*)P, (const uint4*)Q, kscal, (uint4*)out, count);
    PCMM_CUDA_CHECK_LAUNCH();
    return PCMM_OK;
}
