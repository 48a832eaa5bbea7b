"""Bit-exact check of the compression plan (strip codes, ranks, distinct
codes, per-column levels, level-N values and tracking pointers) that the
plan kernel writes, against the definitions of Algorithm 2 computed here
with numpy: level 1 is the sorted set of distinct non-zero values of a
column, level q + 1 the sorted distinct set of the differences of
consecutive level-q values (the first minus zero), and the tracking pointer
of a level-q entry is the position of its difference in level q + 1."""
import numpy as np
import pytest

from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import device, encrypt_gpu
from tests.layout_mirror import NLEV, layout as _layout

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    return device()


def _u16(buf, off, count):
    return np.frombuffer(buf[off:off + 2 * count].tobytes(), dtype=np.uint16)


def _levels(col):
    lev = [np.unique(col[col != 0]).astype(np.int64)]
    ptrs = []
    for _ in range(1, NLEV):
        cur = lev[-1]
        d = np.diff(cur, prepend=0) if len(cur) else cur
        nxt = np.unique(d)
        ptrs.append(np.searchsorted(nxt, d))
        lev.append(nxt)
    return lev, ptrs


@pytest.mark.parametrize("m,n,w,k", [(70, 37, 4, 2), (40, 9, 8, 1), (300, 5, 12, 1), (64, 17, 2, 3),
                                     (2000, 3, 16, 1), (50, 12, 1, 6)])
def test_plan_matches_the_definitions(dev, m, n, w, k):
    pr = inputs.pcmm_problem(3000 + m + w, m, n, 2, w)
    A_h = pr["A"]
    A = pcmm.plaintext16(A_h, dev) if w > 8 else torch.from_numpy(A_h).to(dev)
    ctB = encrypt_gpu(dev, pr)
    ws = pcmm.workspace(m, n, 2, w, k, device=dev)
    pcmm.cussen(A, ctB, 2, w, k=k, ws=ws)
    torch.cuda.synchronize()
    assert pcmm.workspace_status(ws) == 0
    buf = ws.cpu().numpy()
    L = _layout(m, n, w, k)
    A64 = A_h.astype(np.int64)
    for s in range(L["nstrips"]):
        cols = range(s * k, min(s * k + k, n))
        codes = np.zeros(m, dtype=np.int64)
        for t, c in enumerate(cols):
            codes |= A64[:, c] << (w * t)
        distinct = np.unique(codes[codes != 0])
        want_rank = np.where(codes != 0, np.searchsorted(distinct, codes), 0xFFFF)
        got_rank = _u16(buf, L["rank"] + s * m * 2, m)
        assert np.array_equal(got_rank, want_rank), s
        nent = int(np.frombuffer(buf[L["nent"] + 4 * s:L["nent"] + 4 * s + 4].tobytes(), dtype=np.int32)[0])
        assert nent == len(distinct)
        if k > 1:
            got_codes = _u16(buf, L["codes"] + s * L["emax"] * 2, len(distinct))
            assert np.array_equal(got_codes, distinct)
    for c in range(n):
        lev, ptrs = _levels(A64[:, c])
        lens = _u16(buf, L["len"] + c * NLEV * 2, NLEV)
        assert list(lens) == [len(x) for x in lev], c
        vN = _u16(buf, L["vN"] + c * L["l2max"] * 2, len(lev[-1]))
        assert np.array_equal(vN, lev[-1])
        base = L["ptr"] + c * L["ptr_stride"] * 2
        for q in range(NLEV - 1):
            off = base + (0 if q == 0 else (L["n1max"] + (q - 1) * L["l2max"]) * 2)
            got = _u16(buf, off, len(lev[q]))
            assert np.array_equal(got, ptrs[q]), (c, q)
