"""Thin Python binding of ``libpcmm.so`` (declared in ``include/pcmm.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI.  PyTorch provides device memory and the current
CUDA stream.  Device arrays are ``torch.int32`` tensors holding the uint32
words of the quad-planar layouts described in ``include/pcmm.h``.

The library must have been built (``paper_2504_14497_gb300.build.build()``);
there is no fallback: a missing library or a non-zero status raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# The in-tree library; PCMM_LIBRARY may name another build of the same
# sources (for example one compiled with -DPCMM_DEBUG_BOUNDS).
LIB_PATH = os.environ.get("PCMM_LIBRARY") or os.path.join(_HERE, "libpcmm.so")

PCMM_AFF_WORDS = 32
PCMM_JAC_WORDS = 48
PCMM_MAX_WK = 16       # strip code width w * k, bits

# Names of every exported entry point, in the order of include/pcmm.h.
EXPORTS = (
    "pcmm_version", "pcmm_status_string", "pcmm_init", "pcmm_keytable_bytes", "pcmm_keytable",
    "pcmm_encrypt_workspace_bytes", "pcmm_encrypt", "pcmm_encrypt_table", "pcmm_base_mul", "pcmm_bsgs_default_baby", "pcmm_bsgs_bytes", "pcmm_bsgs_build",
    "pcmm_decrypt", "pcmm_schoolbook", "pcmm_schoolbook16", "pcmm_cussen_choose_k",
    "pcmm_workspace_bytes", "pcmm_cussen_workspace_bytes_for", "pcmm_cussen_workspace_bytes", "pcmm_cussen", "pcmm_cussen16", "pcmm_cussen_plan_bytes", "pcmm_cussen_plan", "pcmm_cussen_exec_bytes",
    "pcmm_cussen_execute", "pcmm_cussen_static", "pcmm_strassen_workspace_bytes", "pcmm_strassen", "pcmm_strassen16", "pcmm_batched_workspace_bytes", "pcmm_batched_prepare", "pcmm_batched_run",
    "pcmm_cussen_batched",
    "pcmm_workspace_status", "pcmm_copy_columns", "pcmm_normalize", "pcmm_peak_ops_per_iter",
    "pcmm_peak_threads_per_block", "pcmm_peak_run", "pcmm_profile_enable",
    "pcmm_profile_read", "pcmm_kernel_count", "pcmm_kernel_name", "pcmm_test_wait", "pcmm_test_field",
    "pcmm_test_point",
)

_lock = threading.Lock()
_lib = None


class PcmmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with paper_2504_14497_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, sz, ci, u32p = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)
            sig = {
                "pcmm_version": ([], ci),
                "pcmm_status_string": ([ci], ctypes.c_char_p),
                "pcmm_init": ([ci], ci),
                "pcmm_keytable_bytes": ([], sz),
                "pcmm_keytable": ([u32p, vp, vp], ci),
                "pcmm_encrypt_workspace_bytes": ([], sz),
                "pcmm_encrypt": ([u32p, vp, vp, sz, vp, vp, sz, vp], ci),
                "pcmm_encrypt_table": ([vp, vp, vp, sz, vp, vp], ci),
                "pcmm_base_mul": ([vp, sz, vp, vp], ci),
                "pcmm_bsgs_default_baby": ([ctypes.c_int64], ctypes.c_uint32),
                "pcmm_bsgs_bytes": ([ctypes.c_uint32], sz),
                "pcmm_bsgs_build": ([ctypes.c_uint32, vp, sz, vp], ci),
                "pcmm_decrypt": ([u32p, vp, sz, ctypes.c_int64, ctypes.c_uint32, vp, sz, vp, vp], ci),
                "pcmm_schoolbook": ([vp, ci, ci, ci, vp, ci, vp, vp], ci),
                "pcmm_schoolbook16": ([vp, ci, ci, ci, vp, ci, vp, vp], ci),
                "pcmm_cussen_choose_k": ([ci, ci, ci, ci], ci),
                "pcmm_workspace_bytes": ([ci, ci, ci, ci, ci, ci], sz),
                "pcmm_cussen_workspace_bytes": ([ci, ci, ci, ci, ci], sz),
                "pcmm_cussen_workspace_bytes_for": ([ci, ci, ci, ci, ci, ci], sz),
                "pcmm_cussen": ([vp, ci, ci, ci, vp, ci, vp, ci, vp, sz, vp], ci),
                "pcmm_cussen16": ([vp, ci, ci, ci, vp, ci, vp, ci, vp, sz, vp], ci),
                "pcmm_cussen_plan_bytes": ([ci, ci, ci, ci], sz),
                "pcmm_cussen_plan": ([vp, ci, ci, ci, ci, vp, sz, vp], ci),
                "pcmm_cussen_exec_bytes": ([ci, ci, ci, ci, ci], sz),
                "pcmm_cussen_execute": ([vp, ci, ci, ci, ci, vp, ci, vp, vp, sz, vp], ci),
                "pcmm_cussen_static": ([vp, ci, ci, ci, vp, ci, vp, ci, vp, vp], ci),
                "pcmm_strassen_workspace_bytes": ([ci, ci, ci, ci, ci], sz),
                "pcmm_strassen": ([vp, ci, ci, ci, vp, ci, vp, ci, vp, sz, vp], ci),
                "pcmm_strassen16": ([vp, ci, ci, ci, vp, ci, vp, ci, vp, sz, vp], ci),
                "pcmm_workspace_status": ([vp, u32p, vp], ci),
                "pcmm_batched_workspace_bytes": ([vp, ci, ci], sz),
                "pcmm_batched_prepare": ([vp, ci, ci, vp, sz, vp, vp], ci),
                "pcmm_batched_run": ([vp, vp, vp], ci),
                "pcmm_cussen_batched": ([vp, ci, vp, sz, vp], ci),
                "pcmm_copy_columns": ([vp, sz, sz, vp, sz, sz, sz, sz, vp], ci),
                "pcmm_normalize": ([vp, sz, vp, vp], ci),
                "pcmm_peak_ops_per_iter": ([ci], ci),
                "pcmm_peak_threads_per_block": ([], ci),
                "pcmm_peak_run": ([ci, ci, ci, vp, vp], ci),
                "pcmm_test_field": ([ci, vp, vp, vp, sz, vp], ci),
                "pcmm_test_point": ([ci, vp, vp, vp, vp, sz, vp], ci),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().pcmm_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != 0:
        raise PcmmError(status, what)


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def version() -> int:
    return int(lib().pcmm_version())


def init(device: int = 0):
    _check(lib().pcmm_init(int(device)), "pcmm_init")


# ----------------------------------------------------------------- layouts

def points_to_planar(aos: np.ndarray) -> np.ndarray:
    """uint32[count, 4*Q] point words (coordinates in order) -> [Q, count, 4]."""
    aos = np.ascontiguousarray(aos, dtype=np.uint32)
    count, words = aos.shape
    return np.ascontiguousarray(aos.reshape(count, words // 4, 4).transpose(1, 0, 2))


def planar_to_points(pl: np.ndarray) -> np.ndarray:
    pl = np.asarray(pl, dtype=np.uint32)
    q, count, _ = pl.shape
    return np.ascontiguousarray(pl.transpose(1, 0, 2).reshape(count, 4 * q))


def ct_to_planar(ct: np.ndarray) -> np.ndarray:
    """uint32[..., 2, 16] affine (or [..., 2, 24] Jacobian) ciphertexts ->
    the flat uint32 array of the quad-planar ciphertext layout."""
    ct = np.asarray(ct, dtype=np.uint32)
    words = ct.shape[-1]
    flat = ct.reshape(-1, 2, words)
    count = flat.shape[0]
    pl = flat.reshape(count, 2, words // 4, 4).transpose(1, 2, 0, 3)
    return np.ascontiguousarray(pl).reshape(-1)


def planar_to_ct(flat: np.ndarray, count: int, jacobian: bool = False) -> np.ndarray:
    """Inverse of ct_to_planar: returns uint32[count, 2, 16 or 24]."""
    q = 6 if jacobian else 4
    pl = np.asarray(flat, dtype=np.uint32).reshape(2, q, count, 4)
    return np.ascontiguousarray(pl.transpose(2, 0, 1, 3).reshape(count, 2, 4 * q))


def scalars_to_planar(r: np.ndarray) -> np.ndarray:
    """uint32[..., 8] scalars -> flat quad-planar uint32[8 * count]."""
    r = np.asarray(r, dtype=np.uint32).reshape(-1, 8)
    count = r.shape[0]
    return np.ascontiguousarray(r.reshape(count, 2, 4).transpose(1, 0, 2)).reshape(-1)


def to_device_words(a: np.ndarray, device="cuda"):
    """Host uint32 words -> device int32 tensor (same bits)."""
    torch = _torch()
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).to(device)


def to_host_words(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


# ------------------------------------------------------------- encryption

def keytable_bytes() -> int:
    return int(lib().pcmm_keytable_bytes())


def keytable(H: np.ndarray, device="cuda", stream=None):
    """Comb table of the public key H (uint32[16], x then y)."""
    torch = _torch()
    H = np.ascontiguousarray(H, dtype=np.uint32)
    tab = torch.empty(keytable_bytes(), dtype=torch.uint8, device=device)
    _check(lib().pcmm_keytable(H.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _ptr(tab),
                               _stream(stream)), "pcmm_keytable")
    return tab


def encrypt_workspace_bytes() -> int:
    return int(lib().pcmm_encrypt_workspace_bytes())


def encrypt(H: np.ndarray, msg, r_planar, ws=None, out=None, stream=None):
    """pcmm_encrypt: Enc(b) = (rG, rH + bG) under the public key H
    (uint32[16], x then y, on the host).  msg: cuda uint8[count]; r_planar:
    cuda int32[8 * count] (quad-planar scalars); ws: an optional cuda uint8
    workspace of ``encrypt_workspace_bytes()`` that caches the comb table of
    H between calls.  Returns the affine ciphertext array, cuda
    int32[32 * count]."""
    torch = _torch()
    count = msg.numel()
    if r_planar.numel() != 8 * count:
        raise ValueError("r must hold 8 words per message")
    H = np.ascontiguousarray(H, dtype=np.uint32)
    if ws is None:
        ws = torch.empty(encrypt_workspace_bytes(), dtype=torch.uint8, device=msg.device)
    if out is None:
        out = torch.empty(PCMM_AFF_WORDS * count, dtype=torch.int32, device=msg.device)
    _check(lib().pcmm_encrypt(H.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _ptr(msg), _ptr(r_planar),
                              count, _ptr(out), _ptr(ws), ws.numel(), _stream(stream)), "pcmm_encrypt")
    return out


def encrypt_table(table, msg, r_planar, out=None, stream=None):
    """pcmm_encrypt_table: ``encrypt`` with a key table from ``keytable``."""
    torch = _torch()
    count = msg.numel()
    if r_planar.numel() != 8 * count:
        raise ValueError("r must hold 8 words per message")
    if out is None:
        out = torch.empty(PCMM_AFF_WORDS * count, dtype=torch.int32, device=msg.device)
    _check(lib().pcmm_encrypt_table(_ptr(table), _ptr(msg), _ptr(r_planar), count, _ptr(out),
                                    _stream(stream)), "pcmm_encrypt_table")
    return out


def base_mul(s_planar, count: int, out=None, stream=None):
    """s G for count scalars (cuda int32[8 * count], quad-planar); returns
    the affine point array, cuda int32[16 * count]."""
    torch = _torch()
    if out is None:
        out = torch.empty(16 * count, dtype=torch.int32, device=s_planar.device)
    _check(lib().pcmm_base_mul(_ptr(s_planar), count, _ptr(out), _stream(stream)), "pcmm_base_mul")
    return out


def public_key(sk_words: np.ndarray, device="cuda") -> np.ndarray:
    """KeyGen on the device: H = sk G as host uint32[16] (x then y)."""
    import torch
    s = to_device_words(scalars_to_planar(np.asarray(sk_words, dtype=np.uint32).reshape(1, 8)), device)
    pts = base_mul(s, 1)
    torch.cuda.synchronize()
    return planar_to_points(to_host_words(pts).reshape(4, 1, 4))[0]


# -------------------------------------------------------------- decryption

class BabySteps:
    """Baby-step table j G, j in [1, baby), for decryption by baby-step
    giant-step (independent of the key: one table serves every call with
    messages in [0, mmax] for any mmax)."""

    def __init__(self, baby: int, device="cuda", stream=None):
        torch = _torch()
        L = lib()
        nbytes = int(L.pcmm_bsgs_bytes(int(baby)))
        if nbytes == 0:
            raise ValueError(f"baby = {baby} outside [1, 2^24]")
        self.baby = int(baby)
        self.table = torch.empty(nbytes, dtype=torch.uint8, device=device)
        _check(L.pcmm_bsgs_build(self.baby, _ptr(self.table), nbytes, _stream(stream)),
               "pcmm_bsgs_build")

    @classmethod
    def for_range(cls, mmax: int, device="cuda", stream=None):
        """A table sized by the library's default for messages in [0, mmax]."""
        baby = int(lib().pcmm_bsgs_default_baby(int(mmax)))
        if baby == 0:
            raise ValueError("mmax must be >= 0")
        return cls(baby, device, stream)


def decrypt(sk_words, ct, count: int, mmax: int, steps: BabySteps, out=None, stream=None):
    """Messages of count affine ciphertexts (cuda int32[32 * count]) under
    the secret key sk (uint32[8]): cuda int64[count], -1 where the message is
    outside [0, mmax]."""
    torch = _torch()
    sk = np.ascontiguousarray(np.asarray(sk_words, dtype=np.uint32).reshape(8))
    if ct.numel() < PCMM_AFF_WORDS * count:
        raise ValueError("ct holds fewer than count ciphertexts")
    if out is None:
        out = torch.empty(count, dtype=torch.int64, device=ct.device)
    _check(lib().pcmm_decrypt(sk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), _ptr(ct), int(count),
                              int(mmax), steps.baby, _ptr(steps.table), steps.table.numel(), _ptr(out),
                              _stream(stream)), "pcmm_decrypt")
    return out


# ------------------------------------------------------------------ PC-MM

def _wide(A) -> bool:
    """Whether A holds 16-bit entries (torch int16 or uint16: the bits of a
    uint16 matrix) rather than uint8."""
    es = A.element_size()
    if es not in (1, 2):
        raise TypeError("A must be a uint8 or 16-bit tensor")
    return es == 2


def plaintext16(A_host, device="cuda"):
    """Device copy of a host uint16 matrix, held as int16 (same bits)."""
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(A_host, dtype=np.uint16).view(np.int16)).to(device)


def schoolbook(A, ctB, l: int, w: int, out=None, stream=None):
    """A: cuda uint8[m, n] (w <= 8) or 16-bit [m, n] (w <= 16, see
    ``plaintext16``); ctB: cuda int32[32 * n * l].  Returns the Jacobian
    ciphertext matrix, cuda int32[48 * m * l]."""
    torch = _torch()
    m, n = A.shape
    if out is None:
        out = torch.empty(PCMM_JAC_WORDS * m * l, dtype=torch.int32, device=A.device)
    name = "pcmm_schoolbook16" if _wide(A) else "pcmm_schoolbook"
    _check(getattr(lib(), name)(_ptr(A), m, n, w, _ptr(ctB), l, _ptr(out), _stream(stream)), name)
    return out


def schoolbook16(A, ctB, l: int, w: int, out=None, stream=None):
    """pcmm_schoolbook16: ``schoolbook`` with a 16-bit A."""
    if not _wide(A):
        raise TypeError("schoolbook16 takes a 16-bit A")
    return schoolbook(A, ctB, l, w, out=out, stream=stream)


def choose_k(m: int, n: int, l: int, w: int) -> int:
    return int(lib().pcmm_cussen_choose_k(m, n, l, w))


OP_ENCRYPT, OP_SCHOOLBOOK, OP_CUSSEN, OP_NORMALIZE, OP_CUSSEN_PLAN, OP_CUSSEN_EXEC, OP_STRASSEN = range(7)
WS_INVALID = (1 << (8 * ctypes.sizeof(ctypes.c_size_t))) - 1


def workspace_bytes(op: int, m: int, n: int, l: int, w: int, k: int = 0) -> int:
    """pcmm_workspace_bytes: workspace of one operation (OP_*); WS_INVALID
    for invalid sizes or an unknown operation."""
    return int(lib().pcmm_workspace_bytes(op, m, n, l, w, k))


def cussen_workspace_bytes(m: int, n: int, l: int, w: int, k: int = 0) -> int:
    return int(lib().pcmm_cussen_workspace_bytes(m, n, l, w, k))


def cussen_workspace_bytes_for(m: int, n: int, l: int, w: int, k: int, strips: int) -> int:
    """Workspace bytes with which pcmm_cussen processes `strips` strips per pass."""
    return int(lib().pcmm_cussen_workspace_bytes_for(m, n, l, w, k, strips))


def workspace(m: int, n: int, l: int, w: int, k: int = 0, device="cuda"):
    torch = _torch()
    nb = cussen_workspace_bytes(m, n, l, w, k)
    if nb == 0:
        raise ValueError("invalid PC-MM shape")
    return torch.empty(nb, dtype=torch.uint8, device=device)


def cussen(A, ctB, l: int, w: int, k: int = 0, ws=None, out=None, stream=None):
    """Cussen PC-MM.  Same arguments and result as ``schoolbook`` plus the
    strip width k (0: cost model) and an optional workspace tensor."""
    torch = _torch()
    m, n = A.shape
    if ws is None:
        ws = workspace(m, n, l, w, k, device=A.device)
    if out is None:
        out = torch.empty(PCMM_JAC_WORDS * m * l, dtype=torch.int32, device=A.device)
    name = "pcmm_cussen16" if _wide(A) else "pcmm_cussen"
    _check(getattr(lib(), name)(_ptr(A), m, n, w, _ptr(ctB), l, _ptr(out), k, _ptr(ws), ws.numel(),
                                _stream(stream)), name)
    return out


def cussen16(A, ctB, l: int, w: int, k: int = 0, ws=None, out=None, stream=None):
    """pcmm_cussen16: ``cussen`` with a 16-bit A (entries < 2^w, w <= 16)."""
    if not _wide(A):
        raise TypeError("cussen16 takes a 16-bit A")
    return cussen(A, ctB, l, w, k=k, ws=ws, out=out, stream=stream)


def cussen_static(A, ctB, l: int, w: int, k: int = 0, out=None, status=None, stream=None):
    """Cussen PC-MM on the library's static device scratch (no allocation by
    the library; ``out`` may be passed in so that none happens here either).
    ``status``: an optional cuda int32 tensor of at least one element that
    receives the call's status word (non-zero: the product is invalid).
    Raises PcmmError with PCMM_EUNSUPPORTED when the problem does not fit."""
    torch = _torch()
    m, n = A.shape
    if out is None:
        out = torch.empty(PCMM_JAC_WORDS * m * l, dtype=torch.int32, device=A.device)
    sp = _ptr(status) if status is not None else ctypes.c_void_p(0)
    _check(lib().pcmm_cussen_static(_ptr(A), m, n, w, _ptr(ctB), l, _ptr(out), k, sp, _stream(stream)),
           "pcmm_cussen_static")
    return out


def strassen_workspace_bytes(m: int, n: int, l: int, w: int, levels: int) -> int:
    return int(lib().pcmm_strassen_workspace_bytes(m, n, l, w, levels))


def strassen(A, ctB, l: int, w: int, levels: int, ws=None, out=None, stream=None):
    """pcmm_strassen (uint8 A) or pcmm_strassen16 (16-bit A, see
    ``plaintext16``): Strassen PC-MM with `levels` recursion steps.  ctB:
    cuda int32[32 * n * l]; returns the Jacobian ciphertext matrix, cuda
    int32[48 * m * l]."""
    torch = _torch()
    m, n = A.shape
    if ws is None:
        nb = strassen_workspace_bytes(m, n, l, w, levels)
        if nb == 0:
            raise ValueError("invalid Strassen shape or depth")
        ws = torch.empty(nb, dtype=torch.uint8, device=A.device)
    if out is None:
        out = torch.empty(PCMM_JAC_WORDS * m * l, dtype=torch.int32, device=A.device)
    name = "pcmm_strassen16" if _wide(A) else "pcmm_strassen"
    _check(getattr(lib(), name)(_ptr(A), m, n, w, _ptr(ctB), l, _ptr(out), int(levels), _ptr(ws), ws.numel(),
                                _stream(stream)), name)
    return out


class Problem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int), ("n", ctypes.c_int), ("w", ctypes.c_int),
                ("ctB", ctypes.c_void_p), ("l", ctypes.c_int), ("ctC", ctypes.c_void_p), ("k", ctypes.c_int),
                ("strips", ctypes.c_int)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("nsegs", ctypes.c_int), ("ntasks", ctypes.c_longlong),
                ("nstrips", ctypes.c_longlong), ("nctrs", ctypes.c_int), ("grid", ctypes.c_int),
                ("off_insts", ctypes.c_size_t), ("off_segs", ctypes.c_size_t), ("off_map", ctypes.c_size_t),
                ("off_ctrs", ctypes.c_size_t), ("off_scratch", ctypes.c_size_t),
                ("scratch_u4", ctypes.c_size_t), ("bytes", ctypes.c_size_t)]


class Batch:
    """A prepared batch of Cussen PC-MM instances (one persistent launch).

    items: list of (A cuda uint8 [m, n], ctB cuda int32, l, w, k[, strips per
    pass]); outputs are allocated here (Jacobian, ``self.outs``)."""

    def __init__(self, items, max_strips: int = 0, stream=None):
        torch = _torch()
        L = lib()
        self.items = list(items)
        n = len(self.items)
        self.probs = (Problem * n)()
        self.outs = []
        for i, it in enumerate(self.items):
            A, ctB, l, w, k = it[:5]
            strips = it[5] if len(it) > 5 else 0
            m, nn = A.shape
            out = torch.empty(PCMM_JAC_WORDS * m * l, dtype=torch.int32, device=A.device)
            self.outs.append(out)
            self.probs[i] = Problem(A.data_ptr(), m, nn, w, ctB.data_ptr(), l, out.data_ptr(), k, strips)
        self.max_strips = int(max_strips)
        nb = int(L.pcmm_batched_workspace_bytes(ctypes.cast(self.probs, ctypes.c_void_p), n, self.max_strips))
        if nb == 0:
            raise ValueError("invalid batch")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=self.items[0][0].device)
        self.info = BatchInfo()
        _check(L.pcmm_batched_prepare(ctypes.cast(self.probs, ctypes.c_void_p), n, self.max_strips, _ptr(self.ws), nb,
                                      ctypes.byref(self.info), _stream(stream)), "pcmm_batched_prepare")

    def run(self, stream=None):
        _check(lib().pcmm_batched_run(ctypes.byref(self.info), _ptr(self.ws), _stream(stream)),
               "pcmm_batched_run")
        return self.outs


def problems(items):
    """ctypes array of pcmm_problem for items of (A, ctB, l, w, k, ctC)."""
    arr = (Problem * len(items))()
    for i, (A, ctB, l, w, k, ctC) in enumerate(items):
        m, n = A.shape
        if A.element_size() != 1:
            raise TypeError("batched problems take a uint8 A")
        arr[i] = Problem(_ptr(A).value, m, n, w, _ptr(ctB).value, l, _ptr(ctC).value, k, 0)
    return arr


def batched_workspace_bytes(probs, max_strips: int = 0) -> int:
    return int(lib().pcmm_batched_workspace_bytes(ctypes.cast(probs, ctypes.c_void_p), len(probs),
                                                  int(max_strips)))


def cussen_batched(items, ws=None, stream=None):
    """pcmm_cussen_batched: items of (A, ctB, l, w, k); returns the Jacobian
    outputs (one prepare + run on one workspace)."""
    torch = _torch()
    outs = [torch.empty(PCMM_JAC_WORDS * A.shape[0] * l, dtype=torch.int32, device=A.device)
            for A, _, l, _, _ in items]
    probs = problems([tuple(it) + (o,) for it, o in zip(items, outs)])
    nb = batched_workspace_bytes(probs)
    if nb == 0:
        raise ValueError("invalid batch")
    if ws is None:
        ws = torch.empty(nb, dtype=torch.uint8, device=items[0][0].device)
    _check(lib().pcmm_cussen_batched(ctypes.cast(probs, ctypes.c_void_p), len(probs), _ptr(ws), ws.numel(),
                                     _stream(stream)), "pcmm_cussen_batched")
    return outs


class Plan:
    """A resident Cussen plan of one plaintext matrix A (device memory)."""

    def __init__(self, A, w: int, k: int, stream=None):
        torch = _torch()
        self.m, self.n = A.shape
        self.w, self.k = int(w), int(k)
        nb = int(lib().pcmm_cussen_plan_bytes(self.m, self.n, self.w, self.k))
        if nb == 0:
            raise ValueError("invalid plan shape")
        self.buf = torch.empty(nb, dtype=torch.uint8, device=A.device)
        _check(lib().pcmm_cussen_plan(_ptr(A), self.m, self.n, self.w, self.k, _ptr(self.buf), nb,
                                      _stream(stream)), "pcmm_cussen_plan")

    def exec_bytes(self, l: int) -> int:
        return int(lib().pcmm_cussen_exec_bytes(self.m, self.n, l, self.w, self.k))

    def execute(self, ctB, l: int, ws=None, out=None, stream=None):
        torch = _torch()
        if ws is None:
            ws = torch.empty(self.exec_bytes(l), dtype=torch.uint8, device=ctB.device)
        if out is None:
            out = torch.empty(PCMM_JAC_WORDS * self.m * l, dtype=torch.int32, device=ctB.device)
        _check(lib().pcmm_cussen_execute(_ptr(self.buf), self.m, self.n, self.w, self.k, _ptr(ctB), l,
                                         _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
               "pcmm_cussen_execute")
        return out


def copy_columns(dst, dst_ld: int, dst_col: int, src, src_ld: int, src_col: int, ncols: int,
                 nrows: int, stream=None):
    """Block copy of ncols 16-byte columns over nrows rows (see pcmm.h)."""
    _check(lib().pcmm_copy_columns(_ptr(dst), dst_ld, dst_col, _ptr(src), src_ld, src_col, ncols, nrows,
                                   _stream(stream)), "pcmm_copy_columns")


def workspace_status(ws, stream=None) -> int:
    v = ctypes.c_uint32(0)
    _check(lib().pcmm_workspace_status(_ptr(ws), ctypes.byref(v), _stream(stream)),
           "pcmm_workspace_status")
    return int(v.value)


def normalize(ct_jac, count: int, out=None, stream=None):
    torch = _torch()
    if out is None:
        out = torch.empty(PCMM_AFF_WORDS * count, dtype=torch.int32, device=ct_jac.device)
    _check(lib().pcmm_normalize(_ptr(ct_jac), count, _ptr(out), _stream(stream)), "pcmm_normalize")
    return out


# ---------------------------------------------------------- measurement

PEAK_OPS = {"mad_lo": 0, "mad_hi": 1, "mad_wide": 2, "add_carry": 3, "add": 4, "mul_wide": 5}


def peak_run(op: str, blocks: int, iters: int, sink, stream=None) -> int:
    """Launches the integer-pipe microbenchmark; returns the thread-level
    instructions it executes."""
    code = PEAK_OPS[op]
    _check(lib().pcmm_peak_run(code, int(blocks), int(iters), _ptr(sink), _stream(stream)), "pcmm_peak_run")
    return int(blocks) * int(lib().pcmm_peak_threads_per_block()) * int(iters) * int(
        lib().pcmm_peak_ops_per_iter(code))


# ------------------------------------------------------------- unit tests

def test_wait(ctr, target: int, status, out, warps: int, stream=None):
    L = lib()
    L.pcmm_test_wait.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_int, ctypes.c_void_p]
    L.pcmm_test_wait.restype = ctypes.c_int
    _check(L.pcmm_test_wait(_ptr(ctr), target, _ptr(status), _ptr(out), warps, _stream(stream)),
           "pcmm_test_wait")


def test_field(op: int, a, b=None, stream=None):
    torch = _torch()
    count = a.numel() // 8
    out = torch.empty_like(a)
    bp = _ptr(b) if b is not None else ctypes.c_void_p(0)
    _check(lib().pcmm_test_field(op, _ptr(a), bp, _ptr(out), count, _stream(stream)), "pcmm_test_field")
    return out


def test_point(op: int, P, Q=None, k=None, count: int = 0, stream=None):
    torch = _torch()
    out = torch.empty(16 * count, dtype=torch.int32, device=P.device)
    qp = _ptr(Q) if Q is not None else ctypes.c_void_p(0)
    kp = _ptr(k) if k is not None else ctypes.c_void_p(0)
    _check(lib().pcmm_test_point(op, _ptr(P), qp, kp, _ptr(out), count, _stream(stream)),
           "pcmm_test_point")
    return out


# ---------------------------------------------------------------- profiler

def profile_enable(capacity: int = 8192):
    L = lib()
    L.pcmm_profile_enable.argtypes = [ctypes.c_int]
    L.pcmm_profile_enable.restype = ctypes.c_int
    _check(L.pcmm_profile_enable(int(capacity)), "pcmm_profile_enable")


def profile_read() -> dict:
    """{kernel name: (total ms, launches)} since the last read."""
    L = lib()
    L.pcmm_kernel_count.restype = ctypes.c_int
    L.pcmm_kernel_name.argtypes = [ctypes.c_int]
    L.pcmm_kernel_name.restype = ctypes.c_char_p
    n = int(L.pcmm_kernel_count())
    ms = (ctypes.c_double * n)()
    ln = (ctypes.c_longlong * n)()
    L.pcmm_profile_read.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    L.pcmm_profile_read.restype = ctypes.c_int
    _check(L.pcmm_profile_read(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(ln, ctypes.c_void_p)),
           "pcmm_profile_read")
    return {L.pcmm_kernel_name(i).decode(): (float(ms[i]), int(ln[i])) for i in range(n)}
