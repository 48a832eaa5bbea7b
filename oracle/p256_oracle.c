/*
 * CPU oracle for plaintext-ciphertext matrix multiplication (PC-MM) over
 * EC-ElGamal on NIST P-256 (arXiv 2504.14497).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load, link or
 * call this file: only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Design goal: plain, slow and obviously correct.
 *   - 256-bit integers as 4 x 64-bit little-endian words, products through
 *     unsigned __int128.
 *   - One generic Montgomery (CIOS, R = 2^256) modular arithmetic, used for
 *     both the field prime p and the group order q.  Inversion by Fermat's
 *     little theorem with plain left-to-right square-and-multiply.
 *   - Points in AFFINE coordinates with an explicit infinity flag, textbook
 *     chord-and-tangent group law with every exceptional case spelled out
 *     (Section 2.3: E(F_p) is an abelian group with identity infinity).
 *   - Scalar multiplication of small scalars by the Montgomery ladder
 *     (Algorithm 1); of 256-bit scalars by double-and-add; the closed
 *     form's multiples of G by an 8-bit fixed-base comb whose additions of
 *     one window share a single inversion (Montgomery's simultaneous
 *     inversion), pinned against the bit-by-bit sum.
 *   - Schoolbook PC-MM (Section 3.1), Cussen PC-MM (Algorithms 2 and 3,
 *     N compression levels) and the closed form of the homomorphic linear
 *     combination (Eq. ahe_5_elgamal with H = xG).
 *
 * Every exported function returns 0 on success and a negative value on a
 * bad argument.  External point format: 16 x uint32 little-endian words,
 * x then y, standard (non-Montgomery) representation, fully reduced below
 * p; the point at infinity is all zero words (x = y = 0 is not on the curve
 * because b != 0).  Scalars: 8 x uint32 little-endian words.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Test builds only: -DORC_PLANT=n compiles in one deliberate, plausible
 * mistake (see tests/test_oracle_mutants.py), so that a test can show that
 * the pins catch it.  The oracle proper is built with ORC_PLANT = 0. */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif

typedef unsigned __int128 u128;
typedef struct { uint64_t w[4]; } u256;

/* ------------------------------------------------------------------ */
/* 256-bit unsigned integers                                          */
/* ------------------------------------------------------------------ */

static int hexval(char c) {
    if (c >= '0' && c <= '9') return c - '0';
    if (c >= 'a' && c <= 'f') return c - 'a' + 10;
    if (c >= 'A' && c <= 'F') return c - 'A' + 10;
    return -1;
}

/* Parse exactly 64 hex digits, most significant first. */
static u256 u256_from_hex(const char *s) {
    u256 r; memset(&r, 0, sizeof r);
    for (int i = 0; i < 64; i++) {
        int d = hexval(s[i]);
        int bit = (63 - i) * 4;
        r.w[bit / 64] |= (uint64_t)d << (bit % 64);
    }
    return r;
}

static int u256_cmp(const u256 *a, const u256 *b) {
    for (int i = 3; i >= 0; i--) {
        if (a->w[i] > b->w[i]) return 1;
        if (a->w[i] < b->w[i]) return -1;
    }
    return 0;
}

static int u256_is_zero(const u256 *a) {
    return (a->w[0] | a->w[1] | a->w[2] | a->w[3]) == 0;
}

static uint64_t u256_add(u256 *r, const u256 *a, const u256 *b) {
    u128 c = 0;
    for (int i = 0; i < 4; i++) {
        c += (u128)a->w[i] + b->w[i];
        r->w[i] = (uint64_t)c;
        c >>= 64;
    }
    return (uint64_t)c;
}

static uint64_t u256_sub(u256 *r, const u256 *a, const u256 *b) {
    uint64_t borrow = 0;
    for (int i = 0; i < 4; i++) {
        uint64_t ai = a->w[i], bi = b->w[i];
        uint64_t d = ai - bi - borrow;
        borrow = (ai < bi) || (ai - bi < borrow) ? 1 : 0;
        r->w[i] = d;
    }
    return borrow;
}

static int u256_bit(const u256 *a, int i) { return (int)((a->w[i / 64] >> (i % 64)) & 1); }

static u256 u256_from_u32s(const uint32_t *v) {
    u256 r;
    for (int i = 0; i < 4; i++) r.w[i] = (uint64_t)v[2 * i] | ((uint64_t)v[2 * i + 1] << 32);
    return r;
}

static void u256_to_u32s(const u256 *a, uint32_t *v) {
    for (int i = 0; i < 4; i++) {
        v[2 * i] = (uint32_t)a->w[i];
        v[2 * i + 1] = (uint32_t)(a->w[i] >> 32);
    }
}

static u256 u256_small(uint64_t x) { u256 r; memset(&r, 0, sizeof r); r.w[0] = x; return r; }

/* ------------------------------------------------------------------ */
/* Generic Montgomery arithmetic modulo an odd prime M, R = 2^256      */
/* ------------------------------------------------------------------ */

typedef struct {
    u256 m;        /* the modulus */
    uint64_t minv; /* -M^{-1} mod 2^64 */
    u256 r1;       /* R mod M  (Montgomery form of 1) */
    u256 r2;       /* R^2 mod M */
    u256 mm2;      /* M - 2, the Fermat inversion exponent */
} modctx;

/* x <- 2x mod M, for x < M. */
static void mod_dbl_plain(const modctx *c, u256 *x) {
    u256 t;
    uint64_t carry = u256_add(&t, x, x);
    if (carry || u256_cmp(&t, &c->m) >= 0) u256_sub(&t, &t, &c->m);
    *x = t;
}

static void modctx_init(modctx *c, const char *hex) {
    c->m = u256_from_hex(hex);
    /* Newton iteration for the inverse of the low word modulo 2^64. */
    uint64_t inv = 1;
    for (int i = 0; i < 7; i++) inv *= 2 - c->m.w[0] * inv;
    c->minv = (uint64_t)0 - inv;
    /* R mod M and R^2 mod M by repeated doubling of 1. */
    u256 x = u256_small(1);
    for (int i = 0; i < 256; i++) mod_dbl_plain(c, &x);
    c->r1 = x;
    for (int i = 0; i < 256; i++) mod_dbl_plain(c, &x);
    c->r2 = x;
    u256 two = u256_small(2);
    u256_sub(&c->mm2, &c->m, &two);
}

static void mod_add(const modctx *c, u256 *r, const u256 *a, const u256 *b) {
    u256 t;
    uint64_t carry = u256_add(&t, a, b);
    if (carry || u256_cmp(&t, &c->m) >= 0) u256_sub(&t, &t, &c->m);
    *r = t;
}

static void mod_sub(const modctx *c, u256 *r, const u256 *a, const u256 *b) {
    u256 t;
    uint64_t borrow = u256_sub(&t, a, b);
    if (borrow) u256_add(&t, &t, &c->m);
    *r = t;
}

/* Montgomery product a*b*R^{-1} mod M by coarsely integrated operand
 * scanning (CIOS).  Inputs below M, output below M. */
static void mont_mul(const modctx *c, u256 *r, const u256 *a, const u256 *b) {
    uint64_t t[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 4; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < 4; j++) {
            u128 s = (u128)a->w[j] * b->w[i] + t[j] + carry;
            t[j] = (uint64_t)s;
            carry = (uint64_t)(s >> 64);
        }
        u128 s = (u128)t[4] + carry;
        t[4] = (uint64_t)s;
        t[5] = (uint64_t)(s >> 64);
        uint64_t q = t[0] * c->minv;
        carry = 0;
        for (int j = 0; j < 4; j++) {
            u128 s2 = (u128)q * c->m.w[j] + t[j] + carry;
            t[j] = (uint64_t)s2;
            carry = (uint64_t)(s2 >> 64);
        }
        s = (u128)t[4] + carry;
        t[4] = (uint64_t)s;
        t[5] += (uint64_t)(s >> 64);
        /* t[0] is now zero: divide by 2^64. */
        t[0] = t[1]; t[1] = t[2]; t[2] = t[3]; t[3] = t[4]; t[4] = t[5]; t[5] = 0;
    }
    u256 res = {{t[0], t[1], t[2], t[3]}};
    if (t[4] || u256_cmp(&res, &c->m) >= 0) u256_sub(&res, &res, &c->m);
    *r = res;
}

static void to_mont(const modctx *c, u256 *r, const u256 *a) { mont_mul(c, r, a, &c->r2); }
static void from_mont(const modctx *c, u256 *r, const u256 *a) {
    u256 one = u256_small(1);
    mont_mul(c, r, a, &one);
}

/* a^e for a in Montgomery form; plain left-to-right square-and-multiply. */
static void mont_pow(const modctx *c, u256 *r, const u256 *a, const u256 *e) {
    u256 acc = c->r1;
    for (int i = 255; i >= 0; i--) {
        mont_mul(c, &acc, &acc, &acc);
        if (u256_bit(e, i)) mont_mul(c, &acc, &acc, a);
    }
    *r = acc;
}

/* Inverse by Fermat: a^(M-2), M prime.  a must be non-zero. */
static void mont_inv(const modctx *c, u256 *r, const u256 *a) { mont_pow(c, r, a, &c->mm2); }

/* ------------------------------------------------------------------ */
/* NIST P-256 (FIPS 186-4 D.1.2.3 / SEC 2): y^2 = x^3 - 3x + b over F_p */
/* ------------------------------------------------------------------ */

static modctx FP, FQ;   /* field prime p, group order q */
static u256 CURVE_B;    /* b, Montgomery form mod p */
static u256 THREE_M;    /* 3, Montgomery form mod p */
static u256 GX, GY;     /* generator, Montgomery form mod p */
static int g_ready = 0;

typedef struct { u256 x, y; int inf; } pt;  /* affine, Montgomery-form coordinates */

static void ensure_init(void) {
    if (g_ready) return;
    modctx_init(&FP, "ffffffff00000001000000000000000000000000ffffffffffffffffffffffff");
    modctx_init(&FQ, "ffffffff00000000ffffffffffffffffbce6faada7179e84f3b9cac2fc632551");
    u256 b = u256_from_hex("5ac635d8aa3a93e7b3ebbd55769886bc651d06b0cc53b0f63bce3c3e27d2604b");
    u256 gx = u256_from_hex("6b17d1f2e12c4247f8bce6e563a440f277037d812deb33a0f4a13945d898c296");
    u256 gy = u256_from_hex("4fe342e2fe1a7f9b8ee7eb4a7c0f9e162bce33576b315ececbb6406837bf51f5");
    u256 three = u256_small(3);
    to_mont(&FP, &CURVE_B, &b);
    to_mont(&FP, &GX, &gx);
    to_mont(&FP, &GY, &gy);
    to_mont(&FP, &THREE_M, &three);
    g_ready = 1;
}

static pt pt_inf(void) { pt r; memset(&r, 0, sizeof r); r.inf = 1; return r; }

static pt pt_neg(const pt *a) {
    if (a->inf) return *a;
    pt r = *a;
    u256 zero = u256_small(0);
    mod_sub(&FP, &r.y, &zero, &a->y);
    return r;
}

/* Doubling: lambda = (3x^2 + a) / (2y) with a = -3. */
static pt pt_dbl(const pt *a) {
    if (a->inf || u256_is_zero(&a->y)) return pt_inf();
    u256 x2, num, den, inv, lam, lam2, t, x3, y3;
    mont_mul(&FP, &x2, &a->x, &a->x);
    mont_mul(&FP, &num, &x2, &THREE_M);      /* 3x^2 */
    mod_sub(&FP, &num, &num, &THREE_M);      /* 3x^2 - 3 */
    mod_add(&FP, &den, &a->y, &a->y);        /* 2y */
    mont_inv(&FP, &inv, &den);
    mont_mul(&FP, &lam, &num, &inv);
    mont_mul(&FP, &lam2, &lam, &lam);
    mod_sub(&FP, &x3, &lam2, &a->x);
    mod_sub(&FP, &x3, &x3, &a->x);           /* x3 = lambda^2 - 2x */
    mod_sub(&FP, &t, &a->x, &x3);
    mont_mul(&FP, &y3, &lam, &t);
    mod_sub(&FP, &y3, &y3, &a->y);           /* y3 = lambda (x - x3) - y */
    pt r; r.x = x3; r.y = y3; r.inf = 0;
    return r;
}

/* The chord step of the addition law for finite a, b with x_a != x_b,
 * given dinv = 1 / (x_b - x_a): lambda = (y_b - y_a) dinv. */
static pt pt_chord(const pt *a, const pt *b, const u256 *dinv) {
    u256 num, lam, lam2, t, x3, y3;
    mod_sub(&FP, &num, &b->y, &a->y);
    mont_mul(&FP, &lam, &num, dinv);
    mont_mul(&FP, &lam2, &lam, &lam);
    mod_sub(&FP, &x3, &lam2, &a->x);
    if (ORC_PLANT == 1) mod_add(&FP, &x3, &x3, &b->x);
    else mod_sub(&FP, &x3, &x3, &b->x);      /* x3 = lambda^2 - x1 - x2 */
    mod_sub(&FP, &t, &a->x, &x3);
    mont_mul(&FP, &y3, &lam, &t);
    mod_sub(&FP, &y3, &y3, &a->y);           /* y3 = lambda (x1 - x3) - y1 */
    pt r; r.x = x3; r.y = y3; r.inf = 0;
    return r;
}

/* Addition with all exceptional cases: identity, P = Q, P = -Q. */
static pt pt_add(const pt *a, const pt *b) {
    if (a->inf) return *b;
    if (b->inf) return *a;
    if (u256_cmp(&a->x, &b->x) == 0) {
        if (u256_cmp(&a->y, &b->y) == 0) return ORC_PLANT == 2 ? pt_inf() : pt_dbl(a);
        return pt_inf();                     /* b = -a */
    }
    u256 den, inv;
    mod_sub(&FP, &den, &b->x, &a->x);
    mont_inv(&FP, &inv, &den);
    return pt_chord(a, b, &inv);
}

/* Montgomery ladder, Algorithm 1: exactly t additions and t doublings for
 * a t-bit scalar k (0 <= k < 2^t). */
static pt pt_mul_ladder(uint32_t k, int t, const pt *p) {
    pt r0 = pt_inf(), r1 = *p;
    for (int i = t - 1; i >= 0; i--) {
        int bit = (k >> i) & 1;
        if (bit) { r0 = pt_add(&r1, &r0); r1 = pt_dbl(&r1); }
        else     { r1 = pt_add(&r1, &r0); r0 = pt_dbl(&r0); }
    }
    return r0;
}

/* 256-bit scalar multiplication, left-to-right double-and-add. */
static pt pt_mul_u256(const u256 *s, const pt *p) {
    pt acc = pt_inf();
    for (int i = 255; i >= 0; i--) {
        acc = pt_dbl(&acc);
        if (u256_bit(s, i)) acc = pt_add(&acc, p);
    }
    return acc;
}

static pt generator(void) { pt g; g.x = GX; g.y = GY; g.inf = 0; return g; }

/* 2^i G for i = 0..255, built once by repeated doubling; s G is then the
 * sum of the entries selected by the bits of s. */
static pt G_POW2[256];
static int g_pow2_ready = 0;

static void ensure_pow2(void) {
    ensure_init();
    if (g_pow2_ready) return;
    pt g = generator();
    for (int i = 0; i < 256; i++) { G_POW2[i] = g; g = pt_dbl(&g); }
    g_pow2_ready = 1;
}

static pt pt_mul_base(const u256 *s) {
    pt acc = pt_inf();
    for (int i = 0; i < 256; i++)
        if (u256_bit(s, i)) acc = pt_add(&acc, &G_POW2[i]);
    return acc;
}

/* Fixed-base comb of G with 8-bit windows: COMB_G[i][v] = v 2^(8i) G for
 * windows i = 0..31 and v = 0..255 (v = 0: the identity), built once by
 * repeated addition of 2^(8i) G.  Then s G = sum_i COMB_G[i][byte_i(s)]. */
static pt COMB_G[32][256];
static int g_comb_ready = 0;

static void ensure_comb(void) {
    ensure_pow2();
    if (g_comb_ready) return;
    for (int i = 0; i < 32; i++) {
        COMB_G[i][0] = pt_inf();
        for (int v = 1; v < 256; v++)
            COMB_G[i][v] = pt_add(&COMB_G[i][v - 1], &G_POW2[ORC_PLANT == 6 && i == 5 ? 8 * i + 1 : 8 * i]);
    }
    g_comb_ready = 1;
}

static int scalar_byte(const u256 *s, int i) { return (int)((s->w[i / 8] >> (8 * (i % 8))) & 0xff); }

/* acc[p] = s[p] G for count scalars (COMB_CHUNK at most), window by window.
 * The chord additions of one window share one field inversion (Montgomery's
 * simultaneous inversion: invert the product of all denominators, then peel
 * each 1 / (x_b - x_a) off with two multiplications); additions with the
 * identity or with equal x coordinates go through pt_add. */
#define COMB_CHUNK 256
static void base_mul_comb(const u256 *s, size_t count, pt *acc) {
    u256 den[COMB_CHUNK], pref[COMB_CHUNK];
    int idx[COMB_CHUNK];
    for (size_t p = 0; p < count; p++) acc[p] = pt_inf();
    for (int i = 0; i < 32; i++) {
        int nb = 0;
        for (size_t p = 0; p < count; p++) {
            const int v = scalar_byte(&s[p], i);
            if (!v) continue;
            const pt *T = &COMB_G[i][v];
            if (acc[p].inf || u256_cmp(&acc[p].x, &T->x) == 0) {
                acc[p] = pt_add(&acc[p], T);
                continue;
            }
            mod_sub(&FP, &den[nb], &T->x, &acc[p].x);
            pref[nb] = den[nb];
            if (nb > 0) mont_mul(&FP, &pref[nb], &pref[nb - 1], &den[nb]);
            idx[nb++] = (int)p;
        }
        if (nb == 0) continue;
        u256 inv;                                  /* (den[0] ... den[t])^-1 */
        mont_inv(&FP, &inv, &pref[nb - 1]);
        for (int t = nb - 1; t >= 0; t--) {
            u256 dinv = inv;
            if (t > 0) {
                mont_mul(&FP, &dinv, &inv, &pref[t - 1]);
                mont_mul(&FP, &inv, &inv, &den[t]);
            }
            const int p = idx[t];
            acc[p] = pt_chord(&acc[p], &COMB_G[i][scalar_byte(&s[p], i)], &dinv);
        }
    }
}

static int on_curve(const pt *a) {
    if (a->inf) return 1;
    u256 y2, x2, x3, rhs, t;
    mont_mul(&FP, &y2, &a->y, &a->y);
    mont_mul(&FP, &x2, &a->x, &a->x);
    mont_mul(&FP, &x3, &x2, &a->x);
    mont_mul(&FP, &t, &a->x, &THREE_M);
    mod_sub(&FP, &rhs, &x3, &t);
    mod_add(&FP, &rhs, &rhs, &CURVE_B);
    return u256_cmp(&y2, &rhs) == 0;
}

/* External <-> internal point conversion.  Returns -1 if the external
 * coordinates are not reduced below p. */
static int pt_load(pt *r, const uint32_t *v) {
    u256 x = u256_from_u32s(v), y = u256_from_u32s(v + 8);
    if (u256_is_zero(&x) && u256_is_zero(&y)) { *r = pt_inf(); return 0; }
    if (u256_cmp(&x, &FP.m) >= 0 || u256_cmp(&y, &FP.m) >= 0) return -1;
    to_mont(&FP, &r->x, &x);
    to_mont(&FP, &r->y, &y);
    r->inf = 0;
    return 0;
}

static void pt_store(const pt *a, uint32_t *v) {
    if (a->inf) { memset(v, 0, 16 * sizeof(uint32_t)); return; }
    u256 x, y;
    from_mont(&FP, &x, &a->x);
    from_mont(&FP, &y, &a->y);
    u256_to_u32s(&x, v);
    u256_to_u32s(&y, v + 8);
}

/* ------------------------------------------------------------------ */
/* Exported primitives (pinned by the tests against Python integers    */
/* and against OpenSSL).                                              */
/* ------------------------------------------------------------------ */

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Field and scalar-field ops on canonical standard-form operands.
 * which = 0: mod p, which = 1: mod q.  op: 0 add, 1 sub, 2 mul, 3 inv. */
int orc_mod_op(int which, int op, const uint32_t *a32, const uint32_t *b32, uint32_t *out32) {
    ensure_init();
    const modctx *c = which ? &FQ : &FP;
    u256 a = u256_from_u32s(a32), b = u256_from_u32s(b32), am, bm, r;
    if (u256_cmp(&a, &c->m) >= 0 || u256_cmp(&b, &c->m) >= 0) return -1;
    to_mont(c, &am, &a);
    to_mont(c, &bm, &b);
    switch (op) {
    case 0: mod_add(c, &r, &am, &bm); break;
    case 1: mod_sub(c, &r, &am, &bm); break;
    case 2: mont_mul(c, &r, &am, &bm); break;
    case 3: if (u256_is_zero(&a)) return -1; mont_inv(c, &r, &am); break;
    default: return -1;
    }
    from_mont(c, &r, &r);
    u256_to_u32s(&r, out32);
    return 0;
}

/* Curve constants in standard form: p, q, b, Gx, Gy (5 x 8 words). */
int orc_constants(uint32_t *out) {
    ensure_init();
    u256 v;
    u256_to_u32s(&FP.m, out);
    u256_to_u32s(&FQ.m, out + 8);
    from_mont(&FP, &v, &CURVE_B); u256_to_u32s(&v, out + 16);
    from_mont(&FP, &v, &GX); u256_to_u32s(&v, out + 24);
    from_mont(&FP, &v, &GY); u256_to_u32s(&v, out + 32);
    return 0;
}

int orc_point_add(const uint32_t *P, const uint32_t *Q, uint32_t *out) {
    ensure_init();
    pt a, b;
    if (pt_load(&a, P) || pt_load(&b, Q)) return -1;
    pt r = pt_add(&a, &b);
    pt_store(&r, out);
    return 0;
}

int orc_point_dbl(const uint32_t *P, uint32_t *out) {
    ensure_init();
    pt a;
    if (pt_load(&a, P)) return -1;
    pt r = pt_dbl(&a);
    pt_store(&r, out);
    return 0;
}

int orc_point_neg(const uint32_t *P, uint32_t *out) {
    ensure_init();
    pt a;
    if (pt_load(&a, P)) return -1;
    pt r = pt_neg(&a);
    pt_store(&r, out);
    return 0;
}

/* 1 if on the curve (or infinity), 0 if not, -1 if not reduced. */
int orc_on_curve(const uint32_t *P) {
    ensure_init();
    pt a;
    if (pt_load(&a, P)) return -1;
    return on_curve(&a);
}

/* out = s * P for an arbitrary 256-bit s (double-and-add). */
int orc_scalar_mul(const uint32_t *s32, const uint32_t *P, uint32_t *out) {
    ensure_init();
    pt a;
    if (pt_load(&a, P)) return -1;
    u256 s = u256_from_u32s(s32);
    pt r = pt_mul_u256(&s, &a);
    pt_store(&r, out);
    return 0;
}

/* out = k * P for a t-bit scalar by the Montgomery ladder (Algorithm 1). */
int orc_ladder(uint32_t k, int t, const uint32_t *P, uint32_t *out) {
    ensure_init();
    if (t < 1 || t > 32 || (t < 32 && (k >> t) != 0)) return -1;
    pt a;
    if (pt_load(&a, P)) return -1;
    pt r = pt_mul_ladder(k, t, &a);
    pt_store(&r, out);
    return 0;
}

/* count scalars s_i (8 words each) -> s_i G, using the 2^i G table. */
int orc_base_mul(const uint32_t *s32, size_t count, uint32_t *out) {
    ensure_pow2();
    long long cnt = (long long)count;
#pragma omp parallel for schedule(dynamic, 16)
    for (long long i = 0; i < cnt; i++) {
        u256 s = u256_from_u32s(s32 + 8 * i);
        pt r = pt_mul_base(&s);
        pt_store(&r, out + 16 * i);
    }
    return 0;
}

/* The same products by the fixed-base comb (the evaluation the closed
 * form uses); pinned against orc_base_mul. */
int orc_base_mul_comb(const uint32_t *s32, size_t count, uint32_t *out) {
    ensure_comb();
    long long cnt = (long long)count;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long c0 = 0; c0 < cnt; c0 += COMB_CHUNK) {
        u256 s[COMB_CHUNK];
        pt acc[COMB_CHUNK];
        const size_t n0 = (size_t)(cnt - c0 < COMB_CHUNK ? cnt - c0 : COMB_CHUNK);
        for (size_t t = 0; t < n0; t++) s[t] = u256_from_u32s(s32 + 8 * (c0 + t));
        base_mul_comb(s, n0, acc);
        for (size_t t = 0; t < n0; t++) pt_store(&acc[t], out + 16 * (c0 + t));
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* EC-ElGamal (Section 2.4)                                            */
/* ------------------------------------------------------------------ */

/* KeyGen: H = x G for the secret key x in [1, q-1]. */
int orc_keygen(const uint32_t *sk32, uint32_t *H) {
    ensure_pow2();
    u256 sk = u256_from_u32s(sk32);
    if (u256_is_zero(&sk) || u256_cmp(&sk, &FQ.m) >= 0) return -1;
    pt r = pt_mul_base(&sk);
    pt_store(&r, H);
    return 0;
}

/* Encrypt: (C1, C2) = (r G, r H + phi(m)) with phi(m) = m G.
 * m: count bytes; r: count x 8 words, each in [1, q-1];
 * ct: count x 32 words, C1 (16 words) then C2 (16 words). */
int orc_encrypt(const uint32_t *H32, const uint8_t *msg, const uint32_t *r32, size_t count,
                uint32_t *ct) {
    ensure_pow2();
    pt H;
    if (pt_load(&H, H32)) return -1;
    long long cnt = (long long)count;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(|:bad)
    for (long long i = 0; i < cnt; i++) {
        u256 r = u256_from_u32s(r32 + 8 * i);
        if (u256_is_zero(&r) || u256_cmp(&r, &FQ.m) >= 0) { bad |= 1; continue; }
        pt c1 = pt_mul_base(&r);
        pt rh = pt_mul_u256(&r, &H);
        u256 m = u256_small(msg[i]);
        pt mg = pt_mul_base(&m);
        pt c2 = pt_add(&rh, &mg);
        pt_store(&c1, ct + 32 * i);
        pt_store(&c2, ct + 32 * i + 16);
    }
    return bad ? -1 : 0;
}

/* Decrypt: m = phi^{-1}(C2 - x C1), the discrete log of M = C2 - x C1 to
 * base G found by baby-step giant-step over [0, mmax].  out[i] = -1 when
 * the message is outside the range. */
typedef struct { u256 x, y; uint32_t j; int used; } bsgs_slot;

int orc_decrypt(const uint32_t *sk32, const uint32_t *ct, size_t count, int64_t mmax,
                int64_t *out) {
    ensure_pow2();
    if (mmax < 0) return -1;
    u256 sk = u256_from_u32s(sk32);
    if (u256_is_zero(&sk) || u256_cmp(&sk, &FQ.m) >= 0) return -1;
    uint64_t s = 1;
    while ((s * s) < (uint64_t)mmax + 1) s++;
    /* Baby steps j G, j in [0, s), in an open-addressing table keyed on x. */
    size_t cap = 1;
    while (cap < 2 * s + 2) cap <<= 1;
    bsgs_slot *tab = (bsgs_slot *)calloc(cap, sizeof(bsgs_slot));
    if (!tab) return -2;
    pt g = generator(), jg = pt_inf();
    int have_zero = 0;
    for (uint64_t j = 0; j < s; j++) {
        if (jg.inf) { have_zero = 1; }
        else {
            size_t h = (size_t)(jg.x.w[0] ^ (jg.x.w[1] >> 7)) & (cap - 1);
            while (tab[h].used) h = (h + 1) & (cap - 1);
            tab[h].x = jg.x; tab[h].y = jg.y; tab[h].j = (uint32_t)j; tab[h].used = 1;
        }
        jg = pt_add(&jg, &g);
    }
    (void)have_zero;
    /* Giant stride -s G. */
    u256 sv = u256_small(s);
    pt sg = pt_mul_u256(&sv, &g);
    pt neg_sg = pt_neg(&sg);
    long long cnt = (long long)count;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|:bad)
    for (long long i = 0; i < cnt; i++) {
        pt c1, c2;
        if (pt_load(&c1, ct + 32 * i) || pt_load(&c2, ct + 32 * i + 16)) { bad |= 1; continue; }
        pt xc1 = pt_mul_u256(&sk, &c1);
        pt nx = pt_neg(&xc1);
        pt M = pt_add(&c2, &nx);
        int64_t found = -1;
        for (uint64_t gi = 0; gi * s <= (uint64_t)mmax && found < 0; gi++) {
            if (M.inf) { found = (int64_t)(gi * s); break; }
            size_t h = (size_t)(M.x.w[0] ^ (M.x.w[1] >> 7)) & (cap - 1);
            while (tab[h].used) {
                if (u256_cmp(&tab[h].x, &M.x) == 0 && u256_cmp(&tab[h].y, &M.y) == 0) {
                    found = (int64_t)(gi * s + tab[h].j);
                    break;
                }
                h = (h + 1) & (cap - 1);
            }
            M = ORC_PLANT == 11 ? pt_add(&M, &sg) : pt_add(&M, &neg_sg);
        }
        out[i] = (found >= 0 && found <= mmax) ? found : -1;
    }
    free(tab);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* PC-MM                                                               */
/* Layouts (external): A is m x n uint8 row-major; a ciphertext matrix */
/* with R rows and L columns is R x L x 32 words (C1 then C2 for each   */
/* element, row-major).                                                */
/* ------------------------------------------------------------------ */

typedef struct {
    long long ecsm;        /* scalar multiplications by a non-zero scalar */
    long long ecsm_dbl;    /* doublings executed inside them */
    long long ecsm_add;    /* additions executed inside them */
    long long recon_add;   /* reconstruction / table additions of two finite points */
    long long accum_add;   /* accumulations into C of two finite points */
} orc_counts;

static int load_ct_matrix(pt *dst, const uint32_t *src, size_t count) {
    for (size_t i = 0; i < count; i++) {
        if (pt_load(&dst[2 * i], src + 32 * i)) return -1;
        if (pt_load(&dst[2 * i + 1], src + 32 * i + 16)) return -1;
    }
    return 0;
}

static void store_ct_matrix(uint32_t *dst, const pt *src, size_t count) {
    for (size_t i = 0; i < count; i++) {
        pt_store(&src[2 * i], dst + 32 * i);
        pt_store(&src[2 * i + 1], dst + 32 * i + 16);
    }
}

static int bitlen(uint32_t v) { int t = 0; while (v) { t++; v >>= 1; } return t; }

/* Ladder with operation counting (additions/doublings where both operands
 * are finite are the ones counted as executed). */
static pt ladder_counted(uint32_t k, int t, const pt *p, orc_counts *cnt) {
    pt r0 = pt_inf(), r1 = *p;
    for (int i = t - 1; i >= 0; i--) {
        int bit = (k >> i) & 1;
        pt *ra = (bit ^ (ORC_PLANT == 7)) ? &r0 : &r1;   /* receives r0 + r1 */
        pt *rd = (bit ^ (ORC_PLANT == 7)) ? &r1 : &r0;   /* is doubled */
        if (!r0.inf && !r1.inf) cnt->ecsm_add++;
        if (!rd->inf) cnt->ecsm_dbl++;
        pt s = pt_add(&r1, &r0);
        pt d = pt_dbl(rd);
        *ra = s;
        *rd = d;
    }
    return r0;
}

static pt add_counted(const pt *a, const pt *b, long long *c) {
    if (!a->inf && !b->inf) (*c)++;
    return pt_add(a, b);
}

/* Schoolbook PC-MM (Section 3.1): Enc(c_ij) = sum_k a_ik * Enc(b_kj), each
 * product by the ladder with t = w bits, accumulated by point additions.
 * w is the plaintext bit-width (entries of A must be < 2^w). */
int orc_schoolbook(const uint16_t *A, int m, int n, int l, int w, const uint32_t *ctB,
                   uint32_t *ctC, long long *counts_out) {
    ensure_init();
    if (m < 0 || n < 0 || l < 0 || w < 1 || w > 16) return -1;
    for (long long i = 0; i < (long long)m * n; i++) if (A[i] >> w) return -1;
    pt *B = (pt *)malloc(sizeof(pt) * 2 * (size_t)n * l + 1);
    pt *C = (pt *)malloc(sizeof(pt) * 2 * (size_t)m * l + 1);
    if (!B || !C) { free(B); free(C); return -2; }
    if (load_ct_matrix(B, ctB, (size_t)n * l)) { free(B); free(C); return -1; }
    orc_counts tot; memset(&tot, 0, sizeof tot);
#pragma omp parallel
    {
        orc_counts cnt; memset(&cnt, 0, sizeof cnt);
#pragma omp for schedule(dynamic, 1) collapse(2)
        for (int i = 0; i < m; i++)
            for (int j = 0; j < l; j++)
                for (int c = 0; c < 2; c++) {
                    pt acc = pt_inf();
                    for (int k = 0; k < n; k++) {
                        uint32_t a = A[(size_t)i * n + k];
                        pt term = pt_inf();
                        if (a) {
                            cnt.ecsm++;
                            term = ladder_counted(a, w, &B[2 * ((size_t)k * l + j) + c], &cnt);
                        }
                        acc = add_counted(&acc, &term, &cnt.accum_add);
                    }
                    C[2 * ((size_t)i * l + j) + c] = acc;
                }
#pragma omp critical
        {
            tot.ecsm += cnt.ecsm; tot.ecsm_dbl += cnt.ecsm_dbl; tot.ecsm_add += cnt.ecsm_add;
            tot.recon_add += cnt.recon_add; tot.accum_add += cnt.accum_add;
        }
    }
    store_ct_matrix(ctC, C, (size_t)m * l);
    if (counts_out) {
        counts_out[0] = tot.ecsm; counts_out[1] = tot.ecsm_dbl; counts_out[2] = tot.ecsm_add;
        counts_out[3] = tot.recon_add; counts_out[4] = tot.accum_add;
    }
    free(B); free(C);
    return 0;
}

/* ---- Cussen compression (Algorithm 2), per plaintext vector ---------- */

#define MAXLEV 8

/* Compression plan of one vector of length n0 with N iterations.
 * lev[w] (w = 1..N) holds the level-w vector after sorting and removing
 * duplicates, and for w < N after replacing it by consecutive differences;
 * len[w] is its length; ptr[w][i] (i < len[w-1]) is the tracking pointer:
 * the index in lev[w] of element i of lev[w-1] (level 0 = the input). */
typedef struct {
    int N;
    int len[MAXLEV + 1];
    int32_t *lev[MAXLEV + 1];
    int32_t *ptr[MAXLEV + 1];
} cussen_plan;

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void plan_free(cussen_plan *pl) {
    for (int w = 0; w <= MAXLEV; w++) { free(pl->lev[w]); free(pl->ptr[w]); pl->lev[w] = pl->ptr[w] = NULL; }
}

static int plan_build(cussen_plan *pl, const int32_t *a, int n0, int N) {
    memset(pl, 0, sizeof *pl);
    pl->N = N;
    pl->len[0] = n0;
    pl->lev[0] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n0 + 1));
    if (!pl->lev[0]) return -2;
    memcpy(pl->lev[0], a, sizeof(int32_t) * (size_t)n0);
    for (int w = 1; w <= N; w++) {
        int prev = pl->len[w - 1];
        int32_t *sorted = (int32_t *)malloc(sizeof(int32_t) * (size_t)(prev + 1));
        pl->ptr[w] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(prev + 1));
        if (!sorted || !pl->ptr[w]) { free(sorted); return -2; }
        memcpy(sorted, pl->lev[w - 1], sizeof(int32_t) * (size_t)prev);
        qsort(sorted, (size_t)prev, sizeof(int32_t), cmp_i32);
        /* Eliminate duplicates. */
        int d = 0;
        for (int i = 0; i < prev; i++)
            if (d == 0 || sorted[d - 1] != sorted[i]) sorted[d++] = sorted[i];
        /* Tracking pointers: where each element of the previous level went. */
        for (int i = 0; i < prev; i++) {
            int lo = 0, hi = d - 1, key = pl->lev[w - 1][i];
            while (lo < hi) { int mid = (lo + hi) / 2; if (sorted[mid] < key) lo = mid + 1; else hi = mid; }
            pl->ptr[w][i] = lo;
        }
        /* Differences of consecutive elements except in the last iteration. */
        if (w != N)
            for (int i = d - 1; i >= (ORC_PLANT == 9 ? 2 : 1); i--) sorted[i] = sorted[i] - sorted[i - 1];
        pl->lev[w] = sorted;
        pl->len[w] = d;
    }
    return 0;
}

/* Vector times ciphertext-scalar component by Algorithm 2: out[i] = a_i P.
 * Multiplications by the level-N values use the ladder with t bits. */
static void cussen_apply(const cussen_plan *pl, const pt *P, int t, pt *out, pt *bufA, pt *bufB,
                         orc_counts *cnt) {
    int N = pl->N;
    pt *cur = bufA, *nxt = bufB;
    for (int e = 0; e < pl->len[N]; e++) {
        uint32_t v = (uint32_t)pl->lev[N][e];
        if (v) { cnt->ecsm++; cur[e] = ladder_counted(v, t, P, cnt); }
        else cur[e] = pt_inf();
    }
    for (int w = N; w >= 1; w--) {
        if (w != N)
            for (int i = ORC_PLANT == 3 ? 1 : 0; i + 1 < pl->len[w]; i++)
                cur[i + 1] = add_counted(&cur[i + 1], &cur[i], &cnt->recon_add);
        /* Un-sort and re-insert duplicates into level w-1. */
        pt *dst = (w == 1) ? out : nxt;
        for (int i = 0; i < pl->len[w - 1]; i++)
            dst[i] = cur[(ORC_PLANT == 8 && w == 1 && i == 0) ? pl->len[w] - 1 : pl->ptr[w][i]];
        if (w != 1) { pt *tmp = cur; cur = nxt; nxt = tmp; }
    }
}

/* Cussen PC-MM (Algorithm 3) with N compression iterations, strip width
 * k = 1 exactly as printed.  For strip width k > 1 (an extension that is
 * not in the paper) the columns of each strip are still compressed and
 * reconstructed one by one as above, the distinct k-tuples of the strip
 * are formed by adding the per-column multiples, and every row adds the
 * entry of its tuple once.  Group results are identical for every k. */
int orc_cussen(const uint16_t *A, int m, int n, int l, int w, int kstrip, int N,
               const uint32_t *ctB, uint32_t *ctC, long long *counts_out) {
    ensure_init();
    if (m < 0 || n < 0 || l < 0 || w < 1 || w > 16 || kstrip < 1 || N < 1 || N > MAXLEV) return -1;
    if (w * kstrip > 24) return -1;
    for (long long i = 0; i < (long long)m * n; i++) if (A[i] >> w) return -1;
    pt *B = (pt *)malloc(sizeof(pt) * 2 * (size_t)n * l + 1);
    pt *C = (pt *)malloc(sizeof(pt) * 2 * (size_t)m * l + 1);
    if (!B || !C) { free(B); free(C); return -2; }
    if (load_ct_matrix(B, ctB, (size_t)n * l)) { free(B); free(C); return -1; }
    for (size_t i = 0; i < 2 * (size_t)m * l; i++) C[i] = pt_inf();
    int nstrips = (n + kstrip - 1) / kstrip;
    orc_counts tot; memset(&tot, 0, sizeof tot);
    int err = 0;
    for (int s = 0; s < nstrips && !err; s++) {
        int c0 = s * kstrip, kw = (c0 + kstrip <= n) ? kstrip : n - c0;
        /* Compression of each column of the strip, amortised over all j. */
        cussen_plan plans[32];
        int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
        for (int t = 0; t < kw; t++) {
            for (int i = 0; i < m; i++) col[i] = A[(size_t)i * n + c0 + t];
            if (plan_build(&plans[t], col, m, N)) err = 1;
        }
        free(col);
        /* Distinct tuples of the strip (k > 1 only). */
        int32_t *code = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
        for (int i = 0; i < m; i++) {
            int32_t v = 0;
            for (int t = 0; t < kw; t++) v |= (int32_t)A[(size_t)i * n + c0 + t] << (w * t);
            code[i] = v;
        }
        cussen_plan tp;
        if (kw > 1 && plan_build(&tp, code, m, 1)) err = 1;
        if (!err) {
#pragma omp parallel
            {
                orc_counts cnt; memset(&cnt, 0, sizeof cnt);
                pt *colmul = (pt *)malloc(sizeof(pt) * (size_t)kw * (m + 1));
                pt *bufA = (pt *)malloc(sizeof(pt) * (size_t)(m + 1));
                pt *bufB = (pt *)malloc(sizeof(pt) * (size_t)(m + 1));
                pt *tup = (pt *)malloc(sizeof(pt) * (size_t)(m + 1));
#pragma omp for schedule(dynamic, 1) collapse(2)
                for (int j = 0; j < l; j++)
                    for (int c = 0; c < 2; c++) {
                        for (int t = 0; t < kw; t++)
                            cussen_apply(&plans[t], &B[2 * ((size_t)(c0 + t) * l + j) + c], w,
                                         colmul + (size_t)t * m, bufA, bufB, &cnt);
                        if (kw == 1) {
                            for (int i = 0; i < m; i++) {
                                pt *acc = &C[2 * ((size_t)i * l + j) + c];
                                *acc = add_counted(acc, &colmul[i], &cnt.accum_add);
                            }
                        } else {
                            /* One entry per distinct tuple: the sum of its columns'
                             * multiples, taken from any row that holds the tuple. */
                            int nd = tp.len[1];
                            for (int e = 0; e < nd; e++) tup[e] = pt_inf();
                            int *done = (int *)calloc((size_t)nd + 1, sizeof(int));
                            for (int i = 0; i < m; i++) {
                                int e = tp.ptr[1][i];
                                if (done[e]) continue;
                                done[e] = 1;
                                for (int t = 0; t < kw - (ORC_PLANT == 10); t++)
                                    tup[e] = add_counted(&tup[e], &colmul[(size_t)t * m + i], &cnt.recon_add);
                            }
                            free(done);
                            for (int i = 0; i < m; i++) {
                                pt *acc = &C[2 * ((size_t)i * l + j) + c];
                                *acc = add_counted(acc, &tup[tp.ptr[1][i]], &cnt.accum_add);
                            }
                        }
                    }
                free(colmul); free(bufA); free(bufB); free(tup);
#pragma omp critical
                {
                    tot.ecsm += cnt.ecsm; tot.ecsm_dbl += cnt.ecsm_dbl; tot.ecsm_add += cnt.ecsm_add;
                    tot.recon_add += cnt.recon_add; tot.accum_add += cnt.accum_add;
                }
            }
        }
        for (int t = 0; t < kw; t++) plan_free(&plans[t]);
        if (kw > 1) plan_free(&tp);
        free(code);
    }
    if (!err) store_ct_matrix(ctC, C, (size_t)m * l);
    if (counts_out) {
        counts_out[0] = tot.ecsm; counts_out[1] = tot.ecsm_dbl; counts_out[2] = tot.ecsm_add;
        counts_out[3] = tot.recon_add; counts_out[4] = tot.accum_add;
    }
    free(B); free(C);
    return err ? -2 : 0;
}

/* Closed form of the product (Eq. ahe_5_elgamal with H = x G):
 *   C1_ij = (sum_k a_ik r_kj mod q) G,
 *   C2_ij = (sum_k a_ik (r_kj x + b_kj) mod q) G.
 * Computed for the npairs (i, j) listed in ij (2 ints each); out holds
 * npairs x 32 words.  r: n x l x 8 words; msg: n x l bytes. */
int orc_closed_form(const uint16_t *A, int m, int n, int l, const uint32_t *r32,
                    const uint32_t *sk32, const uint8_t *msg, const int32_t *ij, size_t npairs,
                    uint32_t *out) {
    ensure_comb();
    u256 sk = u256_from_u32s(sk32), skm;
    to_mont(&FQ, &skm, &sk);
    const long long np = (long long)npairs, nl = (long long)n * l;
    /* Per (k, j): r_kj and r_kj x + b_kj mod q, in Montgomery form. */
    u256 *RM = (u256 *)malloc(sizeof(u256) * (size_t)nl);
    u256 *TM = (u256 *)malloc(sizeof(u256) * (size_t)nl);
    u256 *S = (u256 *)malloc(sizeof(u256) * (size_t)(2 * np + 1));
    if (!RM || !TM || !S) { free(RM); free(TM); free(S); return -2; }
#pragma omp parallel for schedule(static)
    for (long long kj = 0; kj < nl; kj++) {
        u256 r = u256_from_u32s(r32 + 8 * kj), b = u256_small(msg[kj]), bm;
        to_mont(&FQ, &RM[kj], &r);
        to_mont(&FQ, &bm, &b);
        mont_mul(&FQ, &TM[kj], &RM[kj], &skm);           /* r x */
        if (ORC_PLANT == 4) mod_sub(&FQ, &TM[kj], &TM[kj], &bm);
        else mod_add(&FQ, &TM[kj], &TM[kj], &bm);        /* r x + b */
    }
    /* Per output: s1 = sum_k a_ik r_kj, s2 = sum_k a_ik (r_kj x + b_kj) mod q.
     * For a plain a < q and a Montgomery-form y R, mont_mul(a, y R) = a y mod
     * q, so the sums come out in plain form. */
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(|:bad)
    for (long long p = 0; p < np; p++) {
        const int i = ij[2 * p], j = ij[2 * p + 1];
        u256 s1 = u256_small(0), s2 = u256_small(0);
        if (i < 0 || i >= m || j < 0 || j >= l) { bad |= 1; S[2 * p] = s1; S[2 * p + 1] = s2; continue; }
        for (int k = 0; k < n; k++) {
            const u256 a = u256_small(A[(size_t)i * n + k]);
            const size_t kj = (size_t)k * l + j;
            u256 t;
            mont_mul(&FQ, &t, &a, &RM[kj]);
            mod_add(&FQ, &s1, &s1, &t);
            mont_mul(&FQ, &t, &a, &TM[kj]);
            mod_add(&FQ, &s2, &s2, &t);
        }
        S[2 * p] = s1;
        S[2 * p + 1] = s2;
    }
    /* C1 = s1 G and C2 = s2 G: scalar 2p goes to words 32p, 2p + 1 to 32p + 16. */
    const long long ns = 2 * np;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long c0 = 0; c0 < ns; c0 += COMB_CHUNK) {
        pt acc[COMB_CHUNK];
        const size_t n0 = (size_t)(ns - c0 < COMB_CHUNK ? ns - c0 : COMB_CHUNK);
        base_mul_comb(S + c0, n0, acc);
        for (size_t t = 0; t < n0; t++) pt_store(&acc[t], out + 16 * (c0 + t));
    }
    free(RM);
    free(TM);
    free(S);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Strassen PC-MM (Section 3.1)                                        */
/* ------------------------------------------------------------------ */

/* a P for a signed plaintext scalar a: |a| P by the ladder (Algorithm 1),
 * negated when a < 0 (block differences of A make negative entries). */
static pt signed_mul(int32_t a, const pt *P, orc_counts *cnt) {
    if (a == 0 || P->inf) return pt_inf();
    uint32_t u = a < 0 ? (uint32_t)(-(int64_t)a) : (uint32_t)a;
    cnt->ecsm++;
    pt r = ladder_counted(u, bitlen(u), P, cnt);
    return a < 0 ? pt_neg(&r) : r;
}

/* r = x + s y for one ciphertext element (both points), s = +1 or -1; the
 * additions of two finite points are counted as block additions. */
static void ct_addsub(pt *r, const pt *x, const pt *y, int s, orc_counts *cnt) {
    for (int c = 0; c < 2; c++) {
        pt yy = s < 0 ? pt_neg(&y[c]) : y[c];
        if (!x[c].inf && !yy.inf) cnt->recon_add++;
        r[c] = pt_add(&x[c], &yy);
    }
}

/* C = A B for a signed plaintext block A (m x n, leading dimension lda)
 * and a ciphertext block B (n x l, ldb elements of two points), C (m x l,
 * ldc).  While levels > 0 and m, n, l are even, one step of Strassen's
 * algorithm: the seven block products
 *   M1 = (A11 + A22)(B11 + B22)   M2 = (A21 + A22) B11
 *   M3 = A11 (B12 - B22)          M4 = A22 (B21 - B11)
 *   M5 = (A11 + A12) B22          M6 = (A21 - A11)(B11 + B12)
 *   M7 = (A12 - A22)(B21 + B22)
 * then C11 = M1 + M4 - M5 + M7, C12 = M3 + M5, C21 = M2 + M4,
 * C22 = M1 - M2 + M3 + M6: 5 plaintext and 5 + 8 = 13 ciphertext block
 * additions or subtractions.  Otherwise the schoolbook product (Section 3.1),
 * one signed scalar multiplication per term and additions into C. */
static void strassen_rec(const int32_t *A, int lda, const pt *B, int ldb, pt *C, int ldc, int m, int n, int l,
                         int levels, orc_counts *cnt, int parallel) {
    if (levels == 0 || (m & 1) || (n & 1) || (l & 1)) {
        for (int i = 0; i < m; i++)
            for (int j = 0; j < l; j++)
                for (int c = 0; c < 2; c++) {
                    pt acc = pt_inf();
                    for (int k = 0; k < n; k++) {
                        pt t = signed_mul(A[(size_t)i * lda + k], &B[2 * ((size_t)k * ldb + j) + c], cnt);
                        if (!acc.inf && !t.inf) cnt->accum_add++;
                        acc = pt_add(&acc, &t);
                    }
                    C[2 * ((size_t)i * ldc + j) + c] = acc;
                }
        return;
    }
    const int mh = m / 2, nh = n / 2, lh = l / 2;
    const size_t sa = (size_t)mh * nh, sb = (size_t)nh * lh, sc = (size_t)mh * lh;
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * 7 * sa);
    pt *T = (pt *)malloc(sizeof(pt) * 2 * 7 * sb);
    pt *M = (pt *)malloc(sizeof(pt) * 2 * 7 * sc);
    for (int i = 0; i < mh; i++)
        for (int k = 0; k < nh; k++) {
            const int32_t a11 = A[(size_t)i * lda + k], a12 = A[(size_t)i * lda + nh + k];
            const int32_t a21 = A[(size_t)(mh + i) * lda + k], a22 = A[(size_t)(mh + i) * lda + nh + k];
            const size_t e = (size_t)i * nh + k;
            S[0 * sa + e] = a11 + a22;
            S[1 * sa + e] = a21 + a22;
            S[2 * sa + e] = a11;
            S[3 * sa + e] = a22;
            S[4 * sa + e] = a11 + a12;
            S[5 * sa + e] = a21 - a11;
            S[6 * sa + e] = a12 - a22;
        }
    for (int k = 0; k < nh; k++)
        for (int j = 0; j < lh; j++) {
            const pt *b11 = &B[2 * ((size_t)k * ldb + j)], *b12 = &B[2 * ((size_t)k * ldb + lh + j)];
            const pt *b21 = &B[2 * ((size_t)(nh + k) * ldb + j)], *b22 = &B[2 * ((size_t)(nh + k) * ldb + lh + j)];
            const size_t e = 2 * ((size_t)k * lh + j);
            ct_addsub(&T[2 * 0 * sb + e], b11, b22, +1, cnt);
            T[2 * 1 * sb + e] = b11[0];
            T[2 * 1 * sb + e + 1] = b11[1];
            ct_addsub(&T[2 * 2 * sb + e], b12, b22, -1, cnt);
            ct_addsub(&T[2 * 3 * sb + e], b21, b11, -1, cnt);
            T[2 * 4 * sb + e] = b22[0];
            T[2 * 4 * sb + e + 1] = b22[1];
            ct_addsub(&T[2 * 5 * sb + e], b11, b12, +1, cnt);
            ct_addsub(&T[2 * 6 * sb + e], b21, b22, +1, cnt);
        }
    if (parallel) {
        orc_counts sub[7];
        memset(sub, 0, sizeof sub);
#pragma omp parallel for schedule(dynamic, 1)
        for (int q = 0; q < 7; q++)
            strassen_rec(S + q * sa, nh, T + 2 * q * sb, lh, M + 2 * q * sc, lh, mh, nh, lh, levels - 1, &sub[q], 0);
        for (int q = 0; q < 7; q++) {
            cnt->ecsm += sub[q].ecsm; cnt->ecsm_dbl += sub[q].ecsm_dbl; cnt->ecsm_add += sub[q].ecsm_add;
            cnt->recon_add += sub[q].recon_add; cnt->accum_add += sub[q].accum_add;
        }
    } else {
        for (int q = 0; q < 7; q++)
            strassen_rec(S + q * sa, nh, T + 2 * q * sb, lh, M + 2 * q * sc, lh, mh, nh, lh, levels - 1, cnt, 0);
    }
    for (int i = 0; i < mh; i++)
        for (int j = 0; j < lh; j++) {
            const size_t e = 2 * ((size_t)i * lh + j);
            const pt *M1 = &M[0 * 2 * sc + e], *M2 = &M[1 * 2 * sc + e], *M3 = &M[2 * 2 * sc + e];
            const pt *M4 = &M[3 * 2 * sc + e], *M5 = &M[4 * 2 * sc + e], *M6 = &M[5 * 2 * sc + e];
            const pt *M7 = &M[6 * 2 * sc + e];
            pt *c11 = &C[2 * ((size_t)i * ldc + j)], *c12 = &C[2 * ((size_t)i * ldc + lh + j)];
            pt *c21 = &C[2 * ((size_t)(mh + i) * ldc + j)], *c22 = &C[2 * ((size_t)(mh + i) * ldc + lh + j)];
            pt t[2];
            ct_addsub(t, M1, M4, +1, cnt);
            ct_addsub(t, t, M5, -1, cnt);
            ct_addsub(c11, t, M7, +1, cnt);
            ct_addsub(c12, M3, M5, +1, cnt);
            ct_addsub(c21, M2, M4, +1, cnt);
            ct_addsub(t, M1, M2, -1, cnt);
            ct_addsub(t, t, M3, +1, cnt);
            ct_addsub(c22, t, M6, ORC_PLANT == 5 ? -1 : +1, cnt);
        }
    free(S);
    free(T);
    free(M);
}

/* Strassen PC-MM of A (m x n, entries < 2^w) and Enc(B) (n x l), `levels`
 * recursion steps (each needs the current m, n, l even), schoolbook below.
 * counts: ecsm (and its ladder's doublings and additions), recon_add =
 * ciphertext block additions/subtractions of two finite points, accum_add
 * = schoolbook accumulations. */
int orc_strassen(const uint16_t *A, int m, int n, int l, int w, int levels, const uint32_t *ctB,
                 uint32_t *ctC, long long *counts) {
    ensure_init();
    if (m < 1 || n < 1 || l < 1 || w < 1 || w > 16 || levels < 0 || levels > 8) return -1;
    const uint32_t amask = (1u << w) - 1u;
    int32_t *Ai = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * n);
    pt *B = (pt *)malloc(sizeof(pt) * 2 * (size_t)n * l);
    pt *C = (pt *)malloc(sizeof(pt) * 2 * (size_t)m * l);
    int rc = 0;
    if (!Ai || !B || !C) rc = -2;
    for (size_t i = 0; rc == 0 && i < (size_t)m * n; i++) {
        if (A[i] & ~amask) rc = -1;
        Ai[i] = A[i];
    }
    if (rc == 0 && load_ct_matrix(B, ctB, (size_t)n * l)) rc = -1;
    if (rc == 0) {
        orc_counts cnt;
        memset(&cnt, 0, sizeof cnt);
        strassen_rec(Ai, n, B, l, C, l, m, n, l, levels, &cnt, 1);
        store_ct_matrix(ctC, C, (size_t)m * l);
        if (counts) {
            counts[0] = cnt.ecsm; counts[1] = cnt.ecsm_dbl; counts[2] = cnt.ecsm_add;
            counts[3] = cnt.recon_add; counts[4] = cnt.accum_add;
        }
    }
    free(Ai);
    free(B);
    free(C);
    return rc;
}
