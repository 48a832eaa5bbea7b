/*
 * pcmm.h - C ABI of libpcmm: plaintext-ciphertext matrix multiplication
 * (PC-MM) with EC-ElGamal over NIST P-256 on one GB300 GPU (sm_103a).
 *
 * Method: arXiv 2504.14497.  A plaintext matrix A (m x n, entries below 2^w)
 * multiplies an element-wise encrypted matrix Enc(B) (n x l), each ciphertext
 * being the pair of curve points (C1, C2) = (rG, rH + bG) (Section 2.4).  The
 * result is Enc(A B): C_ij = sum_k a_ik Enc(b_kj) as point sums
 * (Section 3.1; Eq. ahe_5_elgamal).
 *
 * ---------------------------------------------------------------------------
 * Conventions
 * ---------------------------------------------------------------------------
 * Field elements: 8 x uint32 little-endian limbs, value below p
 *   (p = 2^256 - 2^224 + 2^192 + 2^96 - 1, Section 4.1).
 *
 * Point arrays in device memory are QUAD-PLANAR: for an array of N points,
 *   coordinate quad q (limbs 4q'..4q'+3 of one coordinate) of point i is the
 *   16-byte word at uint32 offset 4 * (q * N + i).
 *   Affine points: 4 quads per point = x[0..3], x[4..7], y[0..3], y[4..7];
 *     infinity is x = y = 0 (not on the curve since b != 0).
 *   Jacobian points (x = X/Z^2, y = Y/Z^3): 6 quads = X lo/hi, Y lo/hi,
 *     Z lo/hi; infinity has Z = 0.
 * Ciphertext arrays of `count` elements are two point arrays, C1 then C2:
 *   affine  : PCMM_AFF_WORDS  = 32 uint32 words per ciphertext,
 *             C1 quads at uint32 offset 0, C2 quads at offset 16 * count;
 *   Jacobian: PCMM_JAC_WORDS  = 48 words per ciphertext,
 *             C1 at offset 0, C2 at offset 24 * count.
 * A matrix of ciphertexts with R rows and L columns is such an array with
 *   count = R * L and element (r, c) at index r * L + c.
 * Scalars (encryption nonces r): quad-planar with 2 quads per scalar
 *   (limbs 0..3, limbs 4..7), 8 words per scalar.
 * The plaintext matrix A: device uint8, row-major m x n, entries < 2^w.
 *
 * Every compute call is asynchronous on the caller's CUDA stream (NULL means
 * the legacy default stream) and allocates no memory: the caller owns all
 * buffers, including the workspace.  Pointers documented as "device" must
 * point to device (or managed) memory of the current device; "host" means
 * host memory.  Argument errors are detected before any launch and return
 * PCMM_EINVAL with nothing enqueued; a failed launch returns PCMM_ECUDA.
 */
#ifndef PCMM_H_
#define PCMM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pcmm_stream_t; /* a cudaStream_t */

typedef enum {
    PCMM_OK = 0,
    PCMM_EINVAL = 1,       /* bad argument (sizes, widths, null pointers)     */
    PCMM_ENOMEM = 2,       /* workspace smaller than required                 */
    PCMM_ECUDA = 3,        /* a CUDA call or kernel launch failed             */
    PCMM_ETIMEOUT = 4,     /* a bounded device-side wait gave up              */
    PCMM_EUNSUPPORTED = 5, /* valid request outside what this build supports */
    PCMM_EDEVICE = 6       /* a kernel flagged bad data (see workspace status) */
} pcmm_status;

#define PCMM_AFF_WORDS 32
#define PCMM_JAC_WORDS 48
#define PCMM_MAX_W 8      /* bit-width w of a uint8 A: 1..8 */
#define PCMM_MAX_W16 16   /* bit-width w of a uint16 A (the paper's t = 12, 16): 1..16 */
#define PCMM_MAX_WK 16    /* strip code width w * k is at most 16 bits */
#define PCMM_N_ITER 4     /* Cussen compression iterations N (Section 3.2) */

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int pcmm_version(void);

/* Human-readable name of a status code (static string, never NULL). */
const char *pcmm_status_string(int status);

/* Builds the fixed-base table of the generator G in static device memory of
 * `device` (makes it current).  Idempotent and cheap after the first call;
 * synchronous.  Must precede pcmm_encrypt on that device.
 * Errors: PCMM_ECUDA if the device cannot be used. */
pcmm_status pcmm_init(int device);

/* ------------------------------------------------------------------------
 * Encryption (Section 2.4): Enc(b) = (rG, rH + bG), phi(b) = bG.
 * Fixed-base comb with one table per 8-bit window: for a base point X,
 * T[i][v] = v 2^(8i) X, i = 0..31, v = 0..255, so that
 * rX = sum_i T[i][byte_i(r)] costs at most 32 mixed additions.
 * ---------------------------------------------------------------------- */

/* Bytes of one key table (the comb table of H). */
size_t pcmm_keytable_bytes(void);

/* Builds the comb table of the public key H.
 * H_host: host, 16 words (x then y), canonical, on the curve, not infinity.
 * keytable: device, pcmm_keytable_bytes() bytes, 16-byte aligned; written.
 * Errors: PCMM_EINVAL (null pointer, H not reduced or infinity). */
pcmm_status pcmm_keytable(const uint32_t *H_host, void *keytable, pcmm_stream_t stream);

/* Bytes of the workspace of pcmm_encrypt: a 256-byte header naming the
 * public key whose comb table follows, then that table. */
size_t pcmm_encrypt_workspace_bytes(void);

/* Encrypts count messages under the public key H (Section 2.4:
 * Enc(b) = (rG, rH + bG), r drawn from [1, q-1] by the caller).
 * H_host: host, 16 words (x then y), canonical, on the curve, not infinity.
 * msg: device uint8[count].  r: device scalars (quad-planar, 8 * count
 * words); each r is used modulo q, and is not checked against [1, q-1].
 * ct: device, affine ciphertext array of count elements (32 * count words),
 * written canonical.
 * ws: device, 256-byte aligned, >= pcmm_encrypt_workspace_bytes() bytes.
 * It caches the comb table of H: a call whose workspace already holds the
 * table of the same H (from an earlier pcmm_encrypt on the same stream
 * order) skips the table build.  Do not write to the workspace between such
 * calls, or clear its first 4 bytes to force a rebuild. Calls that may overlap
 * on the GPU (different streams without an ordering) need separate
 * workspaces: a call with another key rewrites the table in place.  count = 0 only
 * builds (or keeps) the table; msg, r and ct may then be NULL.  Requires
 * pcmm_init on the current device.
 * Errors: PCMM_EINVAL (null or misaligned pointers, H not reduced or
 * infinity, no pcmm_init), PCMM_ENOMEM (ws_bytes too small), PCMM_ECUDA. */
pcmm_status pcmm_encrypt(const uint32_t *H_host, const uint8_t *msg, const uint32_t *r, size_t count,
                         uint32_t *ct, void *ws, size_t ws_bytes, pcmm_stream_t stream);

/* pcmm_encrypt with a key table built once by pcmm_keytable (for callers
 * that keep the table of each key themselves).
 * keytable: device, from pcmm_keytable (read only).  Other arguments as
 * pcmm_encrypt.  Errors: PCMM_EINVAL (null pointers, no pcmm_init),
 * PCMM_ECUDA. */
pcmm_status pcmm_encrypt_table(const void *keytable, const uint8_t *msg, const uint32_t *r, size_t count,
                               uint32_t *ct, pcmm_stream_t stream);

/* Multiplies the generator by count scalars: points[i] = s_i G (KeyGen,
 * Section 2.4: the public key is H = x G for the secret key x).
 * scalars: device, quad-planar (8 * count words), each used modulo q.
 * points: device, affine point array of count points (16 * count words).
 * Requires pcmm_init on the current device.  Errors: PCMM_EINVAL, PCMM_ECUDA. */
pcmm_status pcmm_base_mul(const uint32_t *scalars, size_t count, uint32_t *points,
                          pcmm_stream_t stream);

/* ------------------------------------------------------------------------
 * Decryption (Section 2.4): the key owner recovers m from (C1, C2) as the
 * discrete logarithm of M = C2 - x C1 = m G, searched in [0, mmax] by
 * baby-step giant-step.  A baby-step table holds j G for j in [1, baby)
 * keyed on the affine x coordinate; it does not depend on the key, so one
 * table serves every decryption with the same baby.  Each ciphertext then
 * takes floor(mmax / baby) + 1 giant steps at most.
 * ---------------------------------------------------------------------- */

/* A baby-step count for messages in [0, mmax]: the smallest power of two
 * >= mmax + 1, at least 32 and at most 2^24 (0 if mmax < 0). */
uint32_t pcmm_bsgs_default_baby(int64_t mmax);

/* Bytes of the baby-step table for 1 <= baby <= 2^24 (a hash table of 8-byte
 * slots, at least 2 * baby of them; 0 for an invalid baby). */
size_t pcmm_bsgs_bytes(uint32_t baby);

/* Builds the baby-step table: j G for j in [1, baby).
 * table: device, 16-byte aligned, at least pcmm_bsgs_bytes(baby) bytes;
 * written (cleared first).  Requires pcmm_init on the current device.
 * Errors: PCMM_EINVAL (baby outside [1, 2^24], null or misaligned table, no
 * pcmm_init), PCMM_ENOMEM (table_bytes too small), PCMM_ECUDA. */
pcmm_status pcmm_bsgs_build(uint32_t baby, void *table, size_t table_bytes, pcmm_stream_t stream);

/* Decrypts count ciphertexts: out[i] = m in [0, mmax] with C2 - x C1 = m G,
 * or -1 when no such m exists (the message is outside the range).
 * sk_host: host, 8 words, the secret key x with 1 <= x < q.
 * ct: device, affine ciphertext array of count elements (32 * count words).
 * baby, table: a table built by pcmm_bsgs_build with the same baby (read
 * only).  0 <= mmax <= 2^62.  out: device int64[count], written.
 * Errors: PCMM_EINVAL (null or misaligned pointers, x = 0 or x >= q, mmax
 * out of range, baby outside [1, 2^24], no pcmm_init), PCMM_ENOMEM
 * (table_bytes too small), PCMM_EUNSUPPORTED (mmax / baby >= 2^20: more
 * than 2^20 giant steps per ciphertext; use a larger baby), PCMM_ECUDA. */
pcmm_status pcmm_decrypt(const uint32_t *sk_host, const uint32_t *ct, size_t count, int64_t mmax,
                         uint32_t baby, const void *table, size_t table_bytes, int64_t *out,
                         pcmm_stream_t stream);

/* ------------------------------------------------------------------------
 * PC-MM.  Inputs: A (device uint8 m x n, entries < 2^w), ctB (device affine
 * ciphertext matrix n x l).  Output: ctC (device Jacobian ciphertext matrix
 * m x l, 48 * m * l words), C_ij = sum_k a_ik (B1_kj, B2_kj).
 * ctC must not overlap the inputs.  m, n, l >= 1; 1 <= w <= 8.
 * ---------------------------------------------------------------------- */

/* Schoolbook PC-MM (Section 3.1): every product a_ik B^(kj) by left-to-right
 * double-and-add over the bits of a_ik, then accumulated by point additions.
 * Needs no workspace.  Errors: PCMM_EINVAL, PCMM_ECUDA. */
pcmm_status pcmm_schoolbook(const uint8_t *A, int m, int n, int w, const uint32_t *ctB, int l,
                            uint32_t *ctC, pcmm_stream_t stream);

/* pcmm_schoolbook for plaintext entries of up to 16 bits: A is device uint16
 * m x n (entries < 2^w), 1 <= w <= 16 (the paper's t = 12 and 16 grid,
 * Section 4).  Otherwise as pcmm_schoolbook. */
pcmm_status pcmm_schoolbook16(const uint16_t *A, int m, int n, int w, const uint32_t *ctB, int l,
                              uint32_t *ctC, pcmm_stream_t stream);

/* Strip width chosen by the built-in cost model for a problem shape: the k
 * in [1, 16/w] minimising the modelled work (table build, normalisation and
 * gather, the table work weighted by its lower measured issue efficiency).
 * Accepts 1 <= w <= 16; returns 0 for invalid arguments. */
int pcmm_cussen_choose_k(int m, int n, int l, int w);

/* Workspace bytes with which pcmm_cussen (or pcmm_cussen16) processes
 * `strips` strips per pass (the pass size: table warps of a launch, and the
 * scratch and tables they hold), for strip width k >= 1; 0 for invalid
 * arguments.  strips is capped at the strips of the matrix. */
size_t pcmm_cussen_workspace_bytes_for(int m, int n, int l, int w, int k, int strips);

/* Workspace bytes pcmm_cussen (w <= 8) or pcmm_cussen16 (w <= 16) needs for
 * this shape and strip width k (k = 0: the pcmm_cussen_choose_k value).
 * Returns 0 for invalid arguments.  Larger workspaces let a call process
 * more strips per pass. */
size_t pcmm_cussen_workspace_bytes(int m, int n, int l, int w, int k);

/* Workspace bytes of one operation, by operation code:
 *   PCMM_OP_ENCRYPT     pcmm_encrypt (independent of the sizes);
 *   PCMM_OP_SCHOOLBOOK  pcmm_schoolbook(16): 0, it takes no workspace;
 *   PCMM_OP_CUSSEN      pcmm_cussen / pcmm_cussen16 (k = 0: cost model);
 *   PCMM_OP_NORMALIZE   pcmm_normalize of m * l ciphertexts: 0;
 *   PCMM_OP_CUSSEN_PLAN pcmm_cussen_plan (k = 0: cost model for l);
 *   PCMM_OP_CUSSEN_EXEC pcmm_cussen_execute's default scratch (ditto);
 *   PCMM_OP_STRASSEN    pcmm_strassen with k recursion levels.
 * m x n is the plaintext matrix A, n x l the ciphertext matrix Enc(B), w
 * the bit-width of A's entries (1..16) and k the strip width.  Returns
 * PCMM_WS_INVALID for an unknown operation or invalid sizes (so 0 always
 * means "no workspace needed").  Batched problems are sized by
 * pcmm_batched_workspace_bytes, which takes the problem list. */
#define PCMM_OP_ENCRYPT 0
#define PCMM_OP_SCHOOLBOOK 1
#define PCMM_OP_CUSSEN 2
#define PCMM_OP_NORMALIZE 3
#define PCMM_OP_CUSSEN_PLAN 4
#define PCMM_OP_CUSSEN_EXEC 5
#define PCMM_OP_STRASSEN 6
#define PCMM_WS_INVALID ((size_t)-1)
size_t pcmm_workspace_bytes(int op, int m, int n, int l, int w, int k);

/* Cussen PC-MM (Algorithms 2 and 3).  Strip width k = 1 is Algorithm 3 as
 * printed: each column of A is compressed (sort, remove duplicates, take
 * differences; N = 4 iterations), the compressed values are multiplied by
 * each ciphertext of that row of Enc(B), reconstruction by prefix sums of
 * points rebuilds the multiples of every distinct value, and each output
 * ciphertext adds the multiple its entry selects (the un-sort step fused
 * with the accumulation).  k > 1 (an extension, not in the paper) also
 * combines k adjacent columns into one table of the distinct k-tuples of
 * the strip, so the gather adds once per strip instead of once per column.
 * The result is identical for every k.
 * k: 1 <= k <= 16 / w, or 0 for pcmm_cussen_choose_k.
 * ws: device workspace, 256-byte aligned, of at least
 * pcmm_cussen_workspace_bytes(m, n, l, w, k) bytes; its first 4 bytes are a
 * status word that kernels OR error bits into (1: an entry of A >= 2^w,
 * such entries are masked to w bits; 2: a plan size exceeded its bound;
 * 8, only in a library built with -DPCMM_DEBUG_BOUNDS: a plan index (row
 * rank, tracking pointer, tuple component) outside the table it selects
 * from, the access skipped).  The status word is cleared at the start of
 * every call; read it with pcmm_workspace_status.
 * Errors: PCMM_EINVAL, PCMM_ENOMEM (workspace too small), PCMM_ECUDA. */
pcmm_status pcmm_cussen(const uint8_t *A, int m, int n, int w, const uint32_t *ctB, int l,
                        uint32_t *ctC, int k, void *ws, size_t ws_bytes, pcmm_stream_t stream);

/* pcmm_cussen for plaintext entries of up to 16 bits, the paper's wide
 * values (t = 12 and 16, Sections 3.2 and 4): A is device uint16 m x n with
 * entries < 2^w, 1 <= w <= 16, and 1 <= k <= 16 / w (so k = 1 for w > 8:
 * each column is compressed by the N = 4 difference levels alone, with no
 * table of all 2^w values).  Workspace, status word and errors as
 * pcmm_cussen. */
pcmm_status pcmm_cussen16(const uint16_t *A, int m, int n, int w, const uint32_t *ctB, int l,
                          uint32_t *ctC, int k, void *ws, size_t ws_bytes, pcmm_stream_t stream);

/* The same computation in two phases, so that the plan of a plaintext matrix
 * (it depends on A, w and k only: Algorithm 3 compresses each column of A
 * once for all columns of Enc(B)) can stay resident and serve many Enc(B).
 * pcmm_cussen_plan_bytes: bytes of the plan of an m x n matrix (k >= 1
 *   required), 0 for invalid arguments.
 * pcmm_cussen_plan: builds the plan of A into `plan` (device, 256-byte
 *   aligned, >= pcmm_cussen_plan_bytes), clearing its status word (first 4
 *   bytes; read it with pcmm_workspace_status).
 * pcmm_cussen_exec_bytes: scratch bytes for one execution with l columns
 *   (the default pass: whole waves of table warps on a 152-SM GB300, four
 *   when a pass fits in 16 GiB, else as many as fit, at least one; any
 *   multiple of one strip's need works, larger means fewer passes).
 * pcmm_cussen_execute: ctC = A Enc(B) using a plan built with the same m, n,
 *   w, k (not checked).  The plan is only read, so executions with their own
 *   scratch `ws` may run concurrently on different streams.
 * Errors: PCMM_EINVAL, PCMM_ENOMEM (plan or scratch too small), PCMM_ECUDA. */
size_t pcmm_cussen_plan_bytes(int m, int n, int w, int k);
pcmm_status pcmm_cussen_plan(const uint8_t *A, int m, int n, int w, int k, void *plan,
                             size_t plan_bytes, pcmm_stream_t stream);
size_t pcmm_cussen_exec_bytes(int m, int n, int l, int w, int k);
pcmm_status pcmm_cussen_execute(const void *plan, int m, int n, int w, int k, const uint32_t *ctB,
                                int l, uint32_t *ctC, void *ws, size_t ws_bytes, pcmm_stream_t stream);

/* Cussen PC-MM that allocates nothing, for callers that may not allocate
 * device memory (for instance a plug-in that is only handed its input and
 * output buffers by a framework owning the device memory pool, or a
 * latency-critical loop that cannot afford an allocation's implicit
 * synchronisation).  The paper has no counterpart of this entry point.
 * Same arguments (minus the workspace) and same result as pcmm_cussen.  The
 * scratch space is a fixed 32 MiB array reserved by the library in global
 * memory; every GPU on which the library is loaded holds it until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first
 * call before any stream capture.  All calls on a device share the one
 * array, which keeps the last call's contents: the status word is cleared at
 * the start of every call and everything else is written before it is read,
 * but calls that overlap on the GPU (for instance on two streams without an
 * ordering between them) race on the array and corrupt each other's results.
 * status: NULL, or 4 bytes of device memory (or host memory; pinned keeps
 * the call asynchronous) that receive, in stream order after the kernels,
 * the status word pcmm_cussen would leave in its workspace (1: an entry of
 * A >= 2^w, masked to w bits; 2: a plan size over its bound; 8: a plan index
 * out of range, debug-bounds builds only).  Non-zero means the product is
 * not A Enc(B).
 * The library keeps device state (this array's address, the generator's
 * comb table) per device for the life of the process: a cudaDeviceReset
 * between calls is not supported.
 * Errors: PCMM_EUNSUPPORTED when the problem needs more than the 32 MiB
 * (nothing is launched then), otherwise as pcmm_cussen. */
pcmm_status pcmm_cussen_static(const uint8_t *A, int m, int n, int w, const uint32_t *ctB, int l,
                               uint32_t *ctC, int k, uint32_t *status, pcmm_stream_t stream);

/* Strassen PC-MM (Section 3.1, the paper's second comparison system):
 * `levels` steps of 2 x 2 block recursion, each computing seven block
 * products M1 = (A11 + A22)(B11 + B22), M2 = (A21 + A22) B11,
 * M3 = A11 (B12 - B22), M4 = A22 (B21 - B11), M5 = (A11 + A12) B22,
 * M6 = (A21 - A11)(B11 + B12), M7 = (A12 - A22)(B21 + B22) and
 * C11 = M1 + M4 - M5 + M7, C12 = M3 + M5, C21 = M2 + M4,
 * C22 = M1 - M2 + M3 + M6 (5 plaintext and 13 ciphertext block additions
 * per step), with the schoolbook product of the signed block sums at the
 * leaves.  A, ctB, ctC as pcmm_schoolbook (A uint8, 1 <= w <= 8).
 * levels: 0..7; m, n and l must be multiples of 2^levels.  The block sums
 * of A widen by one bit per step and take both signs; they are held as
 * int16 while w + levels <= 15, else as int32.  ws: device, 256-byte aligned, at least
 * pcmm_strassen_workspace_bytes(m, n, l, w, levels) bytes; its first 4 bytes
 * are a status word (1: an entry of A >= 2^w, masked to w bits), cleared at
 * the start of every call (pcmm_workspace_status reads it).
 * Errors: PCMM_EINVAL (null or misaligned pointers, sizes not multiples of
 * 2^levels, levels or w out of range), PCMM_ENOMEM (workspace too small),
 * PCMM_EUNSUPPORTED (a launch beyond the grid limits), PCMM_ECUDA. */
size_t pcmm_strassen_workspace_bytes(int m, int n, int l, int w, int levels);
pcmm_status pcmm_strassen(const uint8_t *A, int m, int n, int w, const uint32_t *ctB, int l, uint32_t *ctC,
                          int levels, void *ws, size_t ws_bytes, pcmm_stream_t stream);

/* pcmm_strassen for plaintext entries of up to 16 bits (the paper's t = 12
 * and 16): A is device uint16 m x n with entries < 2^w, 1 <= w <= 16.
 * Otherwise as pcmm_strassen (same workspace query). */
pcmm_status pcmm_strassen16(const uint16_t *A, int m, int n, int w, const uint32_t *ctB, int l, uint32_t *ctC,
                            int levels, void *ws, size_t ws_bytes, pcmm_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched PC-MM: many Cussen instances of different shapes and bit-widths
 * in one persistent kernel launch.
 * ---------------------------------------------------------------------- */

/* One instance: A (device uint8 m x n, entries < 2^w), ctB (device affine
 * ciphertext matrix n x l), ctC (device Jacobian output m x l), strip width
 * k (0: pcmm_cussen_choose_k), strips per pass (0: the library's rule, see
 * pcmm_batched_workspace_bytes; > 0: that many, capped by the strips of the
 * instance, by 2 GB per table buffer and by max_strips).  Outputs must not
 * overlap each other or any input. */
typedef struct {
    const uint8_t *A;
    int m, n, w;
    const uint32_t *ctB;
    int l;
    uint32_t *ctC;
    int k;
    int strips;
} pcmm_problem;

/* Launch description written by pcmm_batched_prepare (caller-owned POD). */
typedef struct {
    int count, nsegs;
    long long ntasks, nstrips;
    int nctrs, grid;
    size_t off_insts, off_segs, off_map, off_ctrs, off_scratch, scratch_u4, bytes;
} pcmm_batch_info;

/* Workspace bytes for a batch on the current device (0 for invalid input).
 * max_strips: upper bound on the strips per pass of an instance (its column
 * strips are built and gathered a pass at a time, two passes' tables
 * resident); 0 = the library's choice: at least 1024 table warps per pass
 * (and at least 64 strips while both buffers fit in 256 MB), at most 2 GB
 * per table buffer. */
size_t pcmm_batched_workspace_bytes(const pcmm_problem *probs, int count, int max_strips);

/* Sizes every instance, lays out the workspace (plans, two table buffers per
 * instance, per-warp scratch, counters) and uploads the instance descriptors
 * and the task schedule; synchronises `stream` before returning.  The
 * problems' pointers are baked in: rerun pcmm_batched_prepare when they
 * change.  probs: host array of count problems.  max_strips: as for
 * pcmm_batched_workspace_bytes (same value).  ws: device, 256-byte
 * aligned, >= pcmm_batched_workspace_bytes.  info: host, written.
 * Errors: PCMM_EINVAL, PCMM_ENOMEM, PCMM_ECUDA. */
pcmm_status pcmm_batched_prepare(const pcmm_problem *probs, int count, int max_strips, void *ws,
                                 size_t ws_bytes, pcmm_batch_info *info, pcmm_stream_t stream);

/* Runs a prepared batch: resets the queue and counters (two memsets),
 * builds the plans of all instances (one launch) and runs every table build
 * and gather in ONE persistent kernel whose warps pull tasks from a device
 * queue.  Enqueues a fixed sequence of operations, so it may be captured in a
 * CUDA graph and replayed.  Dependency waits inside the kernel are bounded:
 * if one gives up (about a second), bit 4 of the status word (first 4 bytes
 * of ws, pcmm_workspace_status) is set and the results are invalid.
 * Errors: PCMM_EINVAL, PCMM_ECUDA. */
pcmm_status pcmm_batched_run(const pcmm_batch_info *info, void *ws, pcmm_stream_t stream);

/* Batched Cussen PC-MM in one call (the batched form of Algorithm 3 over
 * many independent problems): pcmm_batched_prepare with the library's
 * default pass sizes, then pcmm_batched_run, on one workspace.  The prepare
 * step uploads the schedule and synchronises `stream`; callers that replay
 * the same batch (for instance from a CUDA graph) should prepare once and
 * call pcmm_batched_run instead.
 * probs: host array of count problems (see pcmm_problem).
 * ws: device, 256-byte aligned, >= pcmm_batched_workspace_bytes(probs,
 * count, 0); its first 4 bytes are the status word of the whole batch.
 * Errors: PCMM_EINVAL, PCMM_ENOMEM, PCMM_EUNSUPPORTED (a queue over 2^31
 * tasks), PCMM_ECUDA. */
pcmm_status pcmm_cussen_batched(const pcmm_problem *probs, int count, void *ws, size_t ws_bytes,
                                pcmm_stream_t stream);

/* Reads the status word of a pcmm_cussen workspace into *status_host after
 * synchronising `stream`.  0 means no kernel raised an error bit. */
pcmm_status pcmm_workspace_status(const void *ws, uint32_t *status_host, pcmm_stream_t stream);

/* Normalises a Jacobian ciphertext array to canonical affine form
 * (Montgomery's simultaneous inversion: each thread takes up to 8
 * ciphertexts, one field inversion per 128-thread block, so per 256 to
 * 2048 points).
 * ct_jac: device, 48 * count words; ct_aff: device, 32 * count words
 * (may not overlap).  Errors: PCMM_EINVAL, PCMM_ECUDA. */
pcmm_status pcmm_normalize(const uint32_t *ct_jac, size_t count, uint32_t *ct_aff,
                           pcmm_stream_t stream);

/* Copies a block of 16-byte words between two row-major matrices of 16-byte
 * words: dst[r * dst_ld + dst_col + c] = src[r * src_ld + src_col + c] for
 * r < nrows, c < ncols (one asynchronous 2-D copy on `stream`).  A quad-planar
 * ciphertext matrix with R rows and L columns is such a matrix with
 * 8 R rows (affine; 12 R if Jacobian) and leading dimension L, so this packs
 * the columns of several Enc(B) into one batch and splits a batched result
 * back.  Errors: PCMM_EINVAL (null pointers, columns out of range), PCMM_ECUDA. */
pcmm_status pcmm_copy_columns(uint32_t *dst, size_t dst_ld, size_t dst_col, const uint32_t *src,
                              size_t src_ld, size_t src_col, size_t ncols, size_t nrows,
                              pcmm_stream_t stream);

/* ------------------------------------------------------------------------
 * Integer-pipe throughput microbenchmark (the measured peaks of the roofline
 * that bounds the PC-MM kernels; not part of the method).  Each of blocks x
 * pcmm_peak_threads_per_block() threads runs eight independent chains of
 * one instruction kind for `iters` iterations, pcmm_peak_ops_per_iter(op)
 * instructions per iteration, so the rate is threads x iters x ops / time.
 * op: PCMM_PEAK_MAD_LO (mad.lo.u32), PCMM_PEAK_MAD_HI (mad.hi.u32),
 * PCMM_PEAK_MAD_WIDE (mad.wide.u32: one 32 x 32 -> 64-bit limb product),
 * PCMM_PEAK_ADD_CARRY (add.cc / addc carry chains), PCMM_PEAK_ADD (add.u32),
 * PCMM_PEAK_MUL_WIDE (mul.wide.u32 chains: one 32 x 32 -> 64-bit product
 * each, multiplicand taken from the previous product).
 * sink: device, 1024 words, practically never written.
 * Errors: PCMM_EINVAL (unknown op, blocks or iters < 1, null sink), PCMM_ECUDA.
 * ---------------------------------------------------------------------- */
#define PCMM_PEAK_MAD_LO 0
#define PCMM_PEAK_MAD_HI 1
#define PCMM_PEAK_MAD_WIDE 2
#define PCMM_PEAK_ADD_CARRY 3
#define PCMM_PEAK_ADD 4
#define PCMM_PEAK_MUL_WIDE 5
int pcmm_peak_ops_per_iter(int op);
int pcmm_peak_threads_per_block(void);
pcmm_status pcmm_peak_run(int op, int blocks, int iters, uint32_t *sink, pcmm_stream_t stream);

/* ------------------------------------------------------------------------
 * Per-kernel timing.  pcmm_profile_enable(capacity > 0) creates `capacity`
 * pairs of CUDA events; from then on every library kernel launch records a
 * start and a stop event on its own stream (until the pool is used up).
 * pcmm_profile_read synchronises those events and writes, for each kernel
 * id 0..pcmm_kernel_count()-1, the summed milliseconds and the number of
 * launches (host arrays of pcmm_kernel_count() entries), then recycles the
 * pool.  pcmm_profile_enable(0) frees the events and disables timing.  Not
 * thread-safe.  Errors: PCMM_EINVAL, PCMM_ECUDA.
 * ---------------------------------------------------------------------- */
pcmm_status pcmm_profile_enable(int capacity);
pcmm_status pcmm_profile_read(double *ms_host, long long *launches_host);
int pcmm_kernel_count(void);
const char *pcmm_kernel_name(int id);

/* ------------------------------------------------------------------------
 * Unit-test entry points for the device arithmetic (device arrays of
 * `count` items, quad-planar like the point arrays).
 * pcmm_test_field: op 0 add, 1 sub, 2 mul, 3 sqr, 4 inv, 5 canonical
 *   form; a, b: 2 quads per element (b unused for ops 3-5); out canonical.
 * pcmm_test_point: op 0 dbl(P), 1 P + Q (mixed: Q affine), 2 P + Q (both
 *   Jacobian), 3 k P for a small scalar k (P affine, k = kscal[i]);
 *   P: Jacobian (6 quads) for ops 0-2, affine (4 quads) for op 3; Q: affine
 *   (op 1) or Jacobian (op 2); out: affine canonical (4 quads).
 * ---------------------------------------------------------------------- */
/* pcmm_test_wait: runs the bounded device-side wait of the persistent batched
 * kernel in `warps` warps (rounded up to a multiple of 4): each waits until
 * *ctr >= target (ctr device int) for at most about a second, then gives up
 * and ORs 4 (timeout) into *status (device); out[w] (device int per warp) is
 * 1 if warp w saw the target, 0 if it gave up. */
pcmm_status pcmm_test_wait(const int *ctr, int target, uint32_t *status, int *out, int warps,
                           pcmm_stream_t stream);
pcmm_status pcmm_test_field(int op, const uint32_t *a, const uint32_t *b, uint32_t *out,
                            size_t count, pcmm_stream_t stream);
pcmm_status pcmm_test_point(int op, const uint32_t *P, const uint32_t *Q, const uint32_t *kscal,
                            uint32_t *out, size_t count, pcmm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* PCMM_H_ */
