"""CPU checks of the boundary: the C-ABI library loads and exports every
function declared in include/pcmm.h (no compute call, no GPU), the host-side
argument validation rejects bad shapes without launching anything, and the
Python layout helpers round-trip."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2504_14497_gb300 import build as pkg_build
from paper_2504_14497_gb300 import pcmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return pcmm.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "pcmm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pcmm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "pcmm_cussen" in names and "pcmm_normalize" in names
    for nm in names:
        assert hasattr(lib, nm), nm
    assert set(pcmm.EXPORTS) <= set(names)


def test_version_and_status_strings(lib):
    assert pcmm.version() >= 10000
    assert pcmm.status_string(0) == "PCMM_OK"
    assert "workspace" in pcmm.status_string(2)
    assert pcmm.status_string(99) == "unknown pcmm status"


def test_host_validation_without_gpu(lib):
    # Invalid shapes are rejected before any CUDA call.
    assert pcmm.cussen_workspace_bytes(0, 4, 4, 4, 1) == 0
    assert pcmm.cussen_workspace_bytes(4, 4, 4, 17, 1) == 0   # w > 16
    assert pcmm.cussen_workspace_bytes(4, 4, 4, 9, 2) == 0    # w * k = 18 > 16
    assert pcmm.cussen_workspace_bytes(4, 4, 4, 4, 5) == 0    # w * k = 20 > 16
    assert pcmm.cussen_workspace_bytes(4, 4, 4, 4, 4) > 0
    assert pcmm.cussen_workspace_bytes(4, 4, 4, 16, 1) > 0
    assert lib.pcmm_cussen(None, 4, 4, 4, None, 4, None, 1, None, 0, None) == 1
    assert lib.pcmm_cussen16(None, 4, 4, 12, None, 4, None, 1, None, 0, None) == 1
    assert lib.pcmm_schoolbook(None, 4, 4, 4, None, 4, None, None) == 1
    assert lib.pcmm_schoolbook16(None, 4, 4, 12, None, 4, None, None) == 1
    # The uint8 entry points reject widths that do not fit a byte (checked
    # before any pointer is used; the dummy pointers are never dereferenced).
    d = ctypes.c_void_p(256)
    assert lib.pcmm_cussen(d, 4, 4, 9, d, 4, d, 1, d, 1 << 20, None) == 1
    assert lib.pcmm_schoolbook(d, 4, 4, 9, d, 4, d, None) == 1
    assert lib.pcmm_cussen16(d, 4, 4, 17, d, 4, d, 1, d, 1 << 20, None) == 1
    assert lib.pcmm_cussen16(d, 4, 4, 9, d, 4, d, 2, d, 1 << 20, None) == 1
    assert lib.pcmm_normalize(None, 4, None, None) == 1


def test_decrypt_host_validation_without_gpu(lib):
    # Baby-step sizing, and arguments rejected before any CUDA call.
    assert lib.pcmm_bsgs_default_baby(-1) == 0
    assert lib.pcmm_bsgs_default_baby(0) == 32
    assert lib.pcmm_bsgs_default_baby(31) == 32
    assert lib.pcmm_bsgs_default_baby(32) == 64
    assert lib.pcmm_bsgs_default_baby(3600) == 4096
    assert lib.pcmm_bsgs_default_baby(1024 * 255 * 255) == 1 << 24
    assert lib.pcmm_bsgs_default_baby(1 << 40) == 1 << 24
    assert lib.pcmm_bsgs_bytes(0) == 0
    assert lib.pcmm_bsgs_bytes((1 << 24) + 1) == 0
    assert lib.pcmm_bsgs_bytes(1) == 16
    assert lib.pcmm_bsgs_bytes(7) == 128
    assert lib.pcmm_bsgs_bytes(32) == 512
    assert lib.pcmm_bsgs_bytes(1 << 24) == 8 << 25
    d = ctypes.c_void_p(256)
    assert lib.pcmm_bsgs_build(0, d, 1 << 20, None) == 1
    assert lib.pcmm_bsgs_build(32, None, 1 << 20, None) == 1
    assert lib.pcmm_bsgs_build(32, ctypes.c_void_p(264), 1 << 20, None) == 1   # misaligned
    assert lib.pcmm_bsgs_build(32, d, 511, None) == 2
    q = 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551

    def key(x):
        return (ctypes.c_uint32 * 8)(*[(x >> (32 * i)) & 0xFFFFFFFF for i in range(8)])

    def dec(x, mmax=100, baby=32, nbytes=512):
        return lib.pcmm_decrypt(key(x), d, 4, mmax, baby, d, nbytes, d, None)

    assert dec(0) == 1
    assert dec(q) == 1
    assert dec(q + 5) == 1
    assert dec(5, mmax=-1) == 1
    assert dec(5, mmax=(1 << 62) + 1) == 1
    assert dec(5, baby=0) == 1
    assert dec(5, baby=(1 << 24) + 1) == 1
    assert dec(5, nbytes=511) == 2
    assert dec(5, mmax=(1 << 20) * 32, baby=32) == 5        # 2^20 + 1 giant steps
    assert dec(5, mmax=1 << 50, baby=1 << 24, nbytes=8 << 25) == 5
    assert dec(q - 1, nbytes=511) == 2
    assert lib.pcmm_decrypt(None, d, 4, 100, 32, d, 512, d, None) == 1


def test_cost_model_choices(lib):
    # Wide values: one column per strip; narrow values: wider strips.
    assert pcmm.choose_k(1024, 1024, 256, 8) == 1
    assert pcmm.choose_k(1024, 1024, 256, 4) >= 2
    assert pcmm.choose_k(1024, 1024, 256, 1) >= 4
    for w in range(1, 17):
        k = pcmm.choose_k(100, 50, 20, w)
        assert 1 <= k and w * k <= 16
    assert pcmm.choose_k(1024, 1024, 256, 12) == 1
    assert pcmm.choose_k(1024, 1024, 256, 16) == 1
    assert pcmm.choose_k(100, 50, 20, 17) == 0


def test_layout_helpers_round_trip():
    rng = np.random.default_rng(0)
    ct = rng.integers(0, 2**32, size=(7, 2, 16), dtype=np.uint64).astype(np.uint32)
    flat = pcmm.ct_to_planar(ct)
    assert flat.shape == (7 * 32,)
    # quad q of C2 of element i sits at word offset 16*count + 4*(q*count + i)
    assert (flat[16 * 7 + 4 * (2 * 7 + 3): 16 * 7 + 4 * (2 * 7 + 3) + 4] == ct[3, 1, 8:12]).all()
    assert (pcmm.planar_to_ct(flat, 7) == ct).all()
    jc = rng.integers(0, 2**32, size=(5, 2, 24), dtype=np.uint64).astype(np.uint32)
    assert (pcmm.planar_to_ct(pcmm.ct_to_planar(jc), 5, jacobian=True) == jc).all()
    r = rng.integers(0, 2**32, size=(6, 8), dtype=np.uint64).astype(np.uint32)
    rp = pcmm.scalars_to_planar(r)
    assert (rp[4 * 6 + 4 * 2: 4 * 6 + 4 * 2 + 4] == r[2, 4:8]).all()


def test_workspace_sizes_follow_the_pass_rule(lib):
    # Host-only: the default workspace is the plan plus one pass of whole
    # waves of table warps (four when a pass fits in 16 GiB, fewer when not,
    # at least one), capped at all strips; mirrored from the documented rule.
    from tests.layout_mirror import PASS_BYTES_CAP, TARGET_WAVES, WAVE_ITEMS, _a256, layout

    for (m, n, l, w, k) in [(1024, 1024, 256, 8, 1), (1024, 1024, 256, 4, 2), (1024, 1024, 256, 16, 1),
                            (2048, 2048, 2048, 3, 2), (6144, 3000, 96, 12, 1), (1024, 700, 256, 1, 6)]:
        L = layout(m, n, w, k, l)
        assert m * 2 * L["njb"] >= 12288          # the gather does not split
        ips = L["items_per_strip"]
        per_strip = ips * L["item_u4"] * 16 + _a256(L["emax"] * 2 * L["lp"] * 64)
        waves = TARGET_WAVES
        while waves > 1 and waves * WAVE_ITEMS // ips > PASS_BYTES_CAP // per_strip:
            waves -= 1
        S = max(1, min(L["nstrips"], waves * WAVE_ITEMS // ips))
        assert pcmm.cussen_workspace_bytes(m, n, l, w, k) == L["plan_bytes"] + S * per_strip, (m, n, l, w, k)


def test_op_workspace_query(lib):
    # pcmm_workspace_bytes dispatches by operation; 0 means "none needed",
    # PCMM_WS_INVALID an invalid request.
    inval = pcmm.WS_INVALID
    assert pcmm.workspace_bytes(pcmm.OP_ENCRYPT, 1, 1, 1, 1) == pcmm.encrypt_workspace_bytes()
    assert pcmm.encrypt_workspace_bytes() == 256 + pcmm.keytable_bytes()
    assert pcmm.workspace_bytes(pcmm.OP_SCHOOLBOOK, 16, 16, 16, 4) == 0
    assert pcmm.workspace_bytes(pcmm.OP_NORMALIZE, 16, 1, 16, 4) == 0
    assert pcmm.workspace_bytes(pcmm.OP_SCHOOLBOOK, 0, 16, 16, 4) == inval
    for (m, n, l, w, k) in [(1024, 1024, 256, 8, 1), (1024, 1024, 256, 4, 0), (300, 70, 9, 12, 1)]:
        assert pcmm.workspace_bytes(pcmm.OP_CUSSEN, m, n, l, w, k) == pcmm.cussen_workspace_bytes(m, n, l, w, k)
        kk = k or pcmm.choose_k(m, n, l, w)
        assert pcmm.workspace_bytes(pcmm.OP_CUSSEN_PLAN, m, n, l, w, k) == lib.pcmm_cussen_plan_bytes(m, n, w, kk)
        assert pcmm.workspace_bytes(pcmm.OP_CUSSEN_EXEC, m, n, l, w, k) == lib.pcmm_cussen_exec_bytes(m, n, l, w, kk)
        # plan + default scratch = the one-call workspace
        assert (pcmm.workspace_bytes(pcmm.OP_CUSSEN_PLAN, m, n, l, w, k)
                + pcmm.workspace_bytes(pcmm.OP_CUSSEN_EXEC, m, n, l, w, k)
                == pcmm.workspace_bytes(pcmm.OP_CUSSEN, m, n, l, w, k))
    assert pcmm.workspace_bytes(pcmm.OP_CUSSEN, 4, 4, 4, 17, 1) == inval
    assert pcmm.workspace_bytes(pcmm.OP_CUSSEN, 4, 4, 4, 4, 5) == inval
    assert pcmm.workspace_bytes(99, 4, 4, 4, 4, 1) == inval
    assert pcmm.workspace_bytes(-1, 4, 4, 4, 4, 1) == inval


def test_encrypt_and_batched_host_validation(lib):
    # Arguments rejected before any CUDA call (dummy pointers never used).
    d = ctypes.c_void_p(256)
    H = (ctypes.c_uint32 * 16)(*([5] * 16))
    nb = pcmm.encrypt_workspace_bytes()
    assert lib.pcmm_encrypt(None, d, d, 4, d, d, nb, None) == 1
    assert lib.pcmm_encrypt((ctypes.c_uint32 * 16)(), d, d, 4, d, d, nb, None) == 1   # infinity
    Hbig = (ctypes.c_uint32 * 16)(*([0xFFFFFFFF] * 16))                                # not reduced
    assert lib.pcmm_encrypt(Hbig, d, d, 4, d, d, nb, None) == 1
    assert lib.pcmm_encrypt(H, None, d, 4, d, d, nb, None) == 1
    assert lib.pcmm_encrypt(H, None, None, 0, None, None, nb, None) == 1              # no workspace
    assert lib.pcmm_encrypt(H, d, d, 4, d, ctypes.c_void_p(272), nb, None) == 1       # misaligned ws
    assert lib.pcmm_encrypt(H, d, d, 4, d, d, nb - 1, None) == 2
    assert lib.pcmm_encrypt_table(None, d, d, 4, d, None) == 1
    assert lib.pcmm_cussen_batched(None, 1, d, 1 << 20, None) == 1
    assert lib.pcmm_cussen_batched(d, 1, None, 1 << 20, None) == 1


def test_static_scratch_holds_the_headline_problem():
    # The allocation-free entry point's 32 MiB scratch holds the plan and one
    # strip of the 1024 x 1024 x 256 product at w = 8 (documented limit).
    from tests.layout_mirror import _a256, layout

    L = layout(1024, 1024, 8, 1, 256)
    assert 1024 * 2 * L["njb"] >= 12288          # the gather does not split
    one_strip = L["items_per_strip"] * L["item_u4"] * 16 + _a256(L["emax"] * 2 * L["lp"] * 64)
    assert L["plan_bytes"] + one_strip <= 32 << 20


def test_strassen_host_validation(lib):
    # Workspace sizing and argument checks, no GPU (dummy pointers unused).
    assert pcmm.strassen_workspace_bytes(16, 16, 16, 4, 0) == 256
    assert pcmm.strassen_workspace_bytes(16, 16, 16, 4, 1) > 256
    assert pcmm.strassen_workspace_bytes(16, 12, 16, 4, 3) == 0      # 12 not a multiple of 8
    assert pcmm.strassen_workspace_bytes(16, 16, 16, 8, 8) == 0      # more than 7 levels
    assert pcmm.strassen_workspace_bytes(256, 256, 256, 8, 7) > 0    # |block sums| <= 2^7 255 fit int16
    assert pcmm.strassen_workspace_bytes(16, 16, 16, 17, 1) == 0     # at most 16-bit entries
    # int16 block sums while w + levels <= 15, int32 beyond.
    def a256(x):
        return (x + 255) // 256 * 256
    for w, eb in ((14, 2), (16, 4)):
        assert pcmm.strassen_workspace_bytes(16, 16, 16, w, 1) == \
            256 + a256(7 * 64 * eb) + a256(7 * 64 * 128) + a256(7 * 64 * 192)
    assert lib.pcmm_strassen(ctypes.c_void_p(256), 16, 16, 9, ctypes.c_void_p(256), 16, ctypes.c_void_p(256), 1,
                             ctypes.c_void_p(256), 1 << 30, None) == 1   # uint8 A takes w <= 8
    # Level t holds 7^t blocks: plaintext int16, affine and Jacobian ciphertexts.
    m, n, l, d = 64, 32, 16, 2
    want, nodes = 256, 1
    for t in range(1, d + 1):
        nodes *= 7
        for b in (nodes * (m >> t) * (n >> t) * 2, nodes * (n >> t) * (l >> t) * 128,
                  nodes * (m >> t) * (l >> t) * 192):
            want = (want + b + 255) // 256 * 256
    assert pcmm.strassen_workspace_bytes(m, n, l, 4, d) == want
    assert pcmm.workspace_bytes(pcmm.OP_STRASSEN, m, n, l, 4, d) == want
    assert pcmm.workspace_bytes(pcmm.OP_STRASSEN, 16, 12, 16, 4, 3) == pcmm.WS_INVALID
    d8 = ctypes.c_void_p(256)
    assert lib.pcmm_strassen(None, 16, 16, 4, d8, 16, d8, 1, d8, 1 << 30, None) == 1
    assert lib.pcmm_strassen(d8, 16, 12, 4, d8, 16, d8, 3, d8, 1 << 30, None) == 1
    assert lib.pcmm_strassen(d8, 16, 16, 4, d8, 16, d8, 1, ctypes.c_void_p(272), 1 << 30, None) == 1
    assert lib.pcmm_strassen(d8, 16, 16, 4, d8, 16, d8, 1, d8, 300, None) == 2


def test_workspace_for_a_pass_size(lib):
    # plan + S strips of scratch and tables (no partial sums when the gather
    # does not split), capped at the matrix's strips; the default workspace
    # is the one for the default pass.
    from tests.layout_mirror import _a256, layout

    for (m, n, l, w, k) in [(1024, 1024, 256, 8, 1), (1024, 700, 256, 4, 2)]:
        L = layout(m, n, w, k, l)
        per_strip = L["items_per_strip"] * L["item_u4"] * 16 + _a256(L["emax"] * 2 * L["lp"] * 64)
        for S in (1, 7, 100):
            assert pcmm.cussen_workspace_bytes_for(m, n, l, w, k, S) == L["plan_bytes"] + S * per_strip
        assert (pcmm.cussen_workspace_bytes_for(m, n, l, w, k, 10 ** 6)
                == L["plan_bytes"] + L["nstrips"] * per_strip)
        full = pcmm.cussen_workspace_bytes(m, n, l, w, k)
        S0 = (full - L["plan_bytes"]) // per_strip
        assert pcmm.cussen_workspace_bytes_for(m, n, l, w, k, S0) == full
    assert pcmm.cussen_workspace_bytes_for(16, 16, 16, 4, 0, 3) == 0
    assert pcmm.cussen_workspace_bytes_for(16, 16, 16, 4, 1, 0) == 0
