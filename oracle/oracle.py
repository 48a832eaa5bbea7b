"""CPU oracle for EC-ElGamal PC-MM over NIST P-256 (arXiv 2504.14497).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  The product
path (the CUDA library and its Python binding) never imports, links or calls
anything here, and this module imports nothing from the product package.

The arithmetic lives in ``p256_oracle.c`` (plain C, 64-bit limbs, affine
textbook group law); this module is argument marshalling plus the
plaintext-only operation-count model of Cussen's compression (Section 3.2,
Algorithm 2), which works on small integer vectors.

Array conventions (numpy):
  * field elements / scalars: ``uint32[..., 8]`` little-endian words;
  * points: ``uint32[..., 16]`` = x words then y words, infinity = all zero;
  * ciphertexts: ``uint32[..., 2, 16]`` = (C1, C2).
Every function raises ``OracleError`` on a negative C status.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "p256_oracle.c")
# ORACLE_LIBRARY may name another build of the same source (the test that
# compiles deliberate mistakes in with -DORC_PLANT=n); it is used as it is.
_LIB = os.environ.get("ORACLE_LIBRARY") or os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

N_ITER = 4  # compression iterations used throughout Sections 3.2-4.2


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if os.environ.get("ORACLE_LIBRARY"):
        return _LIB
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u16p = ctypes.POINTER(ctypes.c_uint16)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            ll = ctypes.POINTER(ctypes.c_longlong)
            sz = ctypes.c_size_t
            ci = ctypes.c_int
            sig = {
                "orc_threads": [],
                "orc_mod_op": [ci, ci, u32p, u32p, u32p],
                "orc_constants": [u32p],
                "orc_point_add": [u32p, u32p, u32p],
                "orc_point_dbl": [u32p, u32p],
                "orc_point_neg": [u32p, u32p],
                "orc_on_curve": [u32p],
                "orc_scalar_mul": [u32p, u32p, u32p],
                "orc_ladder": [ctypes.c_uint32, ci, u32p, u32p],
                "orc_base_mul": [u32p, sz, u32p],
                "orc_base_mul_comb": [u32p, sz, u32p],
                "orc_keygen": [u32p, u32p],
                "orc_encrypt": [u32p, u8p, u32p, sz, u32p],
                "orc_decrypt": [u32p, u32p, sz, ctypes.c_int64, i64p],
                "orc_schoolbook": [u16p, ci, ci, ci, ci, u32p, u32p, ll],
                "orc_cussen": [u16p, ci, ci, ci, ci, ci, ci, u32p, u32p, ll],
                "orc_closed_form": [u16p, ci, ci, ci, u32p, u32p, u8p, i32p, sz, u32p],
                "orc_strassen": [u16p, ci, ci, ci, ci, ci, u32p, u32p, ll],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ci
            _lib = lib
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _u32(a, shape_tail=None):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    if shape_tail is not None and a.shape[-len(shape_tail):] != tuple(shape_tail):
        raise ValueError(f"expected trailing shape {shape_tail}, got {a.shape}")
    return a


def _check(rc, what):
    if rc < 0:
        raise OracleError(f"{what} failed with status {rc}")


# ---------------------------------------------------------------- integers

def int_to_words(x: int, nwords: int = 8) -> np.ndarray:
    return np.array([(x >> (32 * i)) & 0xFFFFFFFF for i in range(nwords)], dtype=np.uint32)


def words_to_int(w) -> int:
    w = np.asarray(w, dtype=np.uint64)
    return sum(int(v) << (32 * i) for i, v in enumerate(w))


def point_to_ints(P):
    """(x, y) Python ints, or None for infinity."""
    P = np.asarray(P)
    if not P.any():
        return None
    return words_to_int(P[:8]), words_to_int(P[8:16])


def ints_to_point(xy) -> np.ndarray:
    if xy is None:
        return np.zeros(16, dtype=np.uint32)
    return np.concatenate([int_to_words(xy[0]), int_to_words(xy[1])])


def threads() -> int:
    return int(_load().orc_threads())


# ------------------------------------------------------- field and group

def constants() -> dict:
    out = np.zeros(40, dtype=np.uint32)
    _check(_load().orc_constants(_p(out, ctypes.c_uint32)), "constants")
    names = ["p", "q", "b", "Gx", "Gy"]
    return {nm: words_to_int(out[8 * i:8 * i + 8]) for i, nm in enumerate(names)}


def mod_op(which: str, op: str, a: int, b: int = 0) -> int:
    """Field (which='p') or scalar-field (which='q') operation on ints."""
    wi = {"p": 0, "q": 1}[which]
    oi = {"add": 0, "sub": 1, "mul": 2, "inv": 3}[op]
    A, B, out = int_to_words(a), int_to_words(b), np.zeros(8, dtype=np.uint32)
    _check(_load().orc_mod_op(wi, oi, _p(A, ctypes.c_uint32), _p(B, ctypes.c_uint32),
                              _p(out, ctypes.c_uint32)), f"mod_op {which} {op}")
    return words_to_int(out)


def point_add(P, Q) -> np.ndarray:
    P, Q, out = _u32(P, (16,)), _u32(Q, (16,)), np.zeros(16, dtype=np.uint32)
    _check(_load().orc_point_add(_p(P, ctypes.c_uint32), _p(Q, ctypes.c_uint32),
                                 _p(out, ctypes.c_uint32)), "point_add")
    return out


def point_dbl(P) -> np.ndarray:
    P, out = _u32(P, (16,)), np.zeros(16, dtype=np.uint32)
    _check(_load().orc_point_dbl(_p(P, ctypes.c_uint32), _p(out, ctypes.c_uint32)), "point_dbl")
    return out


def point_neg(P) -> np.ndarray:
    P, out = _u32(P, (16,)), np.zeros(16, dtype=np.uint32)
    _check(_load().orc_point_neg(_p(P, ctypes.c_uint32), _p(out, ctypes.c_uint32)), "point_neg")
    return out


def on_curve(P) -> bool:
    P = _u32(P, (16,))
    rc = _load().orc_on_curve(_p(P, ctypes.c_uint32))
    _check(rc, "on_curve")
    return bool(rc)


def scalar_mul(s: int, P) -> np.ndarray:
    S, P, out = int_to_words(s), _u32(P, (16,)), np.zeros(16, dtype=np.uint32)
    _check(_load().orc_scalar_mul(_p(S, ctypes.c_uint32), _p(P, ctypes.c_uint32),
                                  _p(out, ctypes.c_uint32)), "scalar_mul")
    return out


def ladder(k: int, t: int, P) -> np.ndarray:
    P, out = _u32(P, (16,)), np.zeros(16, dtype=np.uint32)
    _check(_load().orc_ladder(k, t, _p(P, ctypes.c_uint32), _p(out, ctypes.c_uint32)), "ladder")
    return out


def base_mul(scalars) -> np.ndarray:
    """scalars uint32[count, 8] -> points uint32[count, 16]."""
    S = _u32(scalars, (8,)).reshape(-1, 8)
    out = np.zeros((S.shape[0], 16), dtype=np.uint32)
    _check(_load().orc_base_mul(_p(S, ctypes.c_uint32), S.shape[0], _p(out, ctypes.c_uint32)),
           "base_mul")
    return out


def base_mul_comb(scalars) -> np.ndarray:
    """base_mul by the fixed-base comb with shared inversions (the
    evaluation closed_form uses)."""
    S = _u32(scalars, (8,)).reshape(-1, 8)
    out = np.zeros((S.shape[0], 16), dtype=np.uint32)
    _check(_load().orc_base_mul_comb(_p(S, ctypes.c_uint32), S.shape[0], _p(out, ctypes.c_uint32)),
           "base_mul_comb")
    return out


def generator() -> np.ndarray:
    c = constants()
    return ints_to_point((c["Gx"], c["Gy"]))


# --------------------------------------------------------------- ElGamal

def keygen(sk) -> np.ndarray:
    """H = sk G (Section 2.4).  sk: uint32[8] or int in [1, q-1]."""
    S = int_to_words(sk) if isinstance(sk, int) else _u32(sk, (8,))
    H = np.zeros(16, dtype=np.uint32)
    _check(_load().orc_keygen(_p(S, ctypes.c_uint32), _p(H, ctypes.c_uint32)), "keygen")
    return H


def encrypt(H, msg, r) -> np.ndarray:
    """Enc(b) = (rG, rH + bG).  msg uint8[...], r uint32[..., 8] -> uint32[..., 2, 16]."""
    msg = np.ascontiguousarray(msg, dtype=np.uint8)
    R = _u32(r, (8,))
    if R.shape[:-1] != msg.shape:
        raise ValueError("r must have shape msg.shape + (8,)")
    H = _u32(H, (16,))
    out = np.zeros(msg.shape + (2, 16), dtype=np.uint32)
    _check(_load().orc_encrypt(_p(H, ctypes.c_uint32), _p(msg, ctypes.c_uint8),
                               _p(R, ctypes.c_uint32), msg.size, _p(out, ctypes.c_uint32)),
           "encrypt")
    return out


def decrypt(sk, ct, mmax: int) -> np.ndarray:
    """Baby-step giant-step decryption over [0, mmax]; -1 where out of range."""
    S = int_to_words(sk) if isinstance(sk, int) else _u32(sk, (8,))
    ct = _u32(ct, (2, 16))
    out = np.zeros(ct.shape[:-2], dtype=np.int64)
    _check(_load().orc_decrypt(_p(S, ctypes.c_uint32), _p(ct, ctypes.c_uint32),
                               int(np.prod(ct.shape[:-2])), int(mmax), _p(out, ctypes.c_int64)),
           "decrypt")
    return out


# ------------------------------------------------------------------ PC-MM

COUNT_KEYS = ("ecsm", "ecsm_dbl", "ecsm_add", "recon_add", "accum_add")


def _plaintext(A) -> np.ndarray:
    """A as contiguous uint16 (entries of up to 16 bits, the paper's t <= 16)."""
    A = np.asarray(A)
    if A.size and (int(A.min()) < 0 or int(A.max()) > 0xFFFF):
        raise ValueError("entries of A must lie in [0, 2^16)")
    return np.ascontiguousarray(A, dtype=np.uint16)


def _pcmm_args(A, ctB):
    A = _plaintext(A)
    ctB = _u32(ctB, (2, 16))
    m, n = A.shape
    if ctB.shape[0] != n:
        raise ValueError("Enc(B) must have n rows")
    return A, ctB, m, n, ctB.shape[1]


def schoolbook(A, ctB, w: int):
    """Schoolbook PC-MM (Section 3.1).  Returns (ctC uint32[m, l, 2, 16], counts)."""
    A, ctB, m, n, l = _pcmm_args(A, ctB)
    out = np.zeros((m, l, 2, 16), dtype=np.uint32)
    cnt = (ctypes.c_longlong * 5)()
    _check(_load().orc_schoolbook(_p(A, ctypes.c_uint16), m, n, l, w, _p(ctB, ctypes.c_uint32),
                                  _p(out, ctypes.c_uint32), cnt), "schoolbook")
    return out, dict(zip(COUNT_KEYS, list(cnt)))


def cussen(A, ctB, w: int, k: int = 1, N: int = N_ITER):
    """Cussen PC-MM (Algorithms 2 and 3); k > 1 is the strip extension."""
    A, ctB, m, n, l = _pcmm_args(A, ctB)
    out = np.zeros((m, l, 2, 16), dtype=np.uint32)
    cnt = (ctypes.c_longlong * 5)()
    _check(_load().orc_cussen(_p(A, ctypes.c_uint16), m, n, l, w, k, N, _p(ctB, ctypes.c_uint32),
                              _p(out, ctypes.c_uint32), cnt), "cussen")
    return out, dict(zip(COUNT_KEYS, list(cnt)))


def strassen(A, ctB, w: int, levels: int):
    """Strassen PC-MM (Section 3.1): `levels` recursion steps of seven block
    products and 13 ciphertext block additions (m, n, l even at each step),
    schoolbook products below.  Returns (ctC uint32[m, l, 2, 16], counts)
    with recon_add = ciphertext block additions, accum_add = schoolbook
    accumulations."""
    A, ctB, m, n, l = _pcmm_args(A, ctB)
    out = np.zeros((m, l, 2, 16), dtype=np.uint32)
    cnt = (ctypes.c_longlong * 5)()
    _check(_load().orc_strassen(_p(A, ctypes.c_uint16), m, n, l, w, levels, _p(ctB, ctypes.c_uint32),
                                _p(out, ctypes.c_uint32), cnt), "strassen")
    return out, dict(zip(COUNT_KEYS, list(cnt)))


def closed_form(A, r, sk, msg, pairs=None) -> np.ndarray:
    """C_ij = ((sum_k a_ik r_kj) G, (sum_k a_ik (r_kj sk + b_kj)) G).

    ``pairs``: int array [P, 2] of (i, j); default all m*l outputs, returned
    as uint32[m, l, 2, 16]; with pairs, uint32[P, 2, 16]."""
    A = _plaintext(A)
    m, n = A.shape
    R = _u32(r, (8,))
    l = R.shape[1]
    msg = np.ascontiguousarray(msg, dtype=np.uint8)
    S = int_to_words(sk) if isinstance(sk, int) else _u32(sk, (8,))
    full = pairs is None
    if full:
        ii, jj = np.meshgrid(np.arange(m), np.arange(l), indexing="ij")
        pairs = np.stack([ii.ravel(), jj.ravel()], axis=1)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32)
    out = np.zeros((pairs.shape[0], 2, 16), dtype=np.uint32)
    _check(_load().orc_closed_form(_p(A, ctypes.c_uint16), m, n, l, _p(R, ctypes.c_uint32),
                                   _p(S, ctypes.c_uint32), _p(msg, ctypes.c_uint8),
                                   _p(pairs, ctypes.c_int32), pairs.shape[0],
                                   _p(out, ctypes.c_uint32)), "closed_form")
    return out.reshape(m, l, 2, 16) if full else out


# ------------------------------------------- operation-count model (Sec. 3)

def compress_counts(vec, N: int = N_ITER):
    """Multiplications and additions of Cussen's vector-scalar algorithm
    (Algorithm 2) for one plaintext vector, as the paper counts them
    (Appendix tables): a zero entry contributes the identity and costs
    nothing.  mults = non-zero entries of the level-N vector; adds = sum
    over levels 1..N-1 of the non-zero entries of the level vector."""
    v = np.asarray(vec, dtype=np.int64)
    adds = 0
    for w in range(1, N + 1):
        v = np.unique(v)  # sort ascending, eliminate duplicates
        if w != N:
            d = v.copy()
            d[1:] = v[1:] - v[:-1]  # consecutive differences
            adds += int(np.count_nonzero(d))
            v = d
    return int(np.count_nonzero(v)), adds


def ct_vector_equiv(mults: float, adds: float, t: int) -> float:
    """Equivalent point additions of a plaintext vector times one ciphertext
    (Section 3.3): 2 components x (ECSM ~ 2t additions per multiply + adds)."""
    return 2 * (2 * t * mults + adds)


def pcmm_equiv_cussen(n: int, vec_equiv: float) -> float:
    """Square PC-MM (m = n = l): n*l vector-times-ciphertext products plus
    2*m*l*(n-1) accumulation additions."""
    return n * n * vec_equiv + 2 * n * n * (n - 1)


def pcmm_equiv_strassen(n: int, t: int) -> int:
    """Equivalent point additions of Strassen PC-MM of square n x n
    matrices (n a power of two) recursed down to single entries (Section
    3.1): 7^log2(n) plaintext-ciphertext products of two ECSMs each (2t
    additions per ECSM, Section 3.3) plus 13 ciphertext block additions per
    step of two points each, A(n) = 7 A(n/2) + 13 (n/2)^2."""
    mults, adds, k = 1, 0, 1
    while k < n:
        adds = 7 * adds + 13 * k * k
        mults *= 7
        k *= 2
    return mults * 2 * 2 * t + 2 * adds


def pcmm_equiv_schoolbook(n: int, t: int) -> int:
    """2 n^3 ECSMs of 2t equivalent additions plus 2 n^2 (n-1) additions."""
    return 2 * n ** 3 * 2 * t + 2 * n * n * (n - 1)
