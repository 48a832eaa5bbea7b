"""The strip tables the table kernel builds and normalises (Algorithm 2's
reconstruction, Algorithm 3 steps 5-6; canonical affine entries), read back
from the workspace and checked entry by entry against the oracle: the entry
of rank e of strip s, component c and output column j is the e-th smallest
distinct non-zero code of the strip, u, times the ciphertexts of the strip's
columns, sum_t u_t B_c^(s k + t, j)."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import device, encrypt_gpu
from tests.layout_mirror import layout, single_pass_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.mark.parametrize("w,k", [(8, 1), (4, 2), (2, 3), (12, 1)])
def test_strip_tables_match_the_oracle(dev, w, k):
    m, n, l = 3072, 2 * k + 1, 64                 # ragged last strip for k > 1
    pr = inputs.pcmm_problem(4000 + w, m, n, l, w)
    A_h = pr["A"]
    A = pcmm.plaintext16(A_h, dev) if w > 8 else torch.from_numpy(A_h).to(dev)
    ctB = encrypt_gpu(dev, pr)
    L = layout(m, n, w, k, l)
    ws = pcmm.workspace(m, n, l, w, k, device=dev)
    pcmm.cussen(A, ctB, l, w, k=k, ws=ws)
    torch.cuda.synchronize()
    assert pcmm.workspace_status(ws) == 0
    buf = ws.cpu().numpy()
    toff, tpoints = single_pass_table(L)
    words = np.frombuffer(buf[toff:toff + tpoints * 64].tobytes(), dtype=np.uint32).reshape(4, tpoints, 4)
    ct = oracle.encrypt(oracle.keygen(pr["sk"]), pr["B"], pr["r"])     # [n, l, 2, 16]
    rng = np.random.default_rng(w * 10 + k)
    A64 = A_h.astype(np.int64)
    mask = (1 << w) - 1
    for s in range(L["nstrips"]):
        cols = list(range(s * k, min(s * k + k, n)))
        codes = np.zeros(m, dtype=np.int64)
        for t, c in enumerate(cols):
            codes |= A64[:, c] << (w * t)
        distinct = np.unique(codes[codes != 0])
        for e in list(rng.integers(0, len(distinct), 5)) + [0, len(distinct) - 1]:
            u = int(distinct[e])
            for c in (0, 1):
                for j in (int(rng.integers(0, l)), l - 1):
                    want = np.zeros(16, dtype=np.uint32)
                    for t, col in enumerate(cols):
                        ut = (u >> (w * t)) & mask
                        if ut:
                            want = oracle.point_add(want, oracle.scalar_mul(ut, ct[col, j, c]))
                    idx = ((s * L["emax"] + e) * 2 + c) * L["lp"] + j
                    got = np.concatenate([words[q, idx] for q in range(4)])
                    assert np.array_equal(got, want), (s, e, c, j)


@pytest.mark.parametrize("w,k", [(8, 1), (4, 2), (2, 3), (12, 1)])
def test_every_strip_table_entry(dev, w, k):
    """Every entry of every strip table (all distinct codes u, both
    components, all l columns) against the closed form of the entry:
    component 1 is (sum_t u_t r_t) G and component 2 (sum_t u_t (r_t x +
    b_t)) G, since B = (r G, r H + b G) with H = x G."""
    Q = 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551
    m, n, l = 3072, 2 * k + 1, 64
    pr = inputs.pcmm_problem(4100 + w, m, n, l, w)
    A_h = pr["A"]
    A = pcmm.plaintext16(A_h, dev) if w > 8 else torch.from_numpy(A_h).to(dev)
    ctB = encrypt_gpu(dev, pr)
    L = layout(m, n, w, k, l)
    ws = pcmm.workspace(m, n, l, w, k, device=dev)
    pcmm.cussen(A, ctB, l, w, k=k, ws=ws)
    torch.cuda.synchronize()
    assert pcmm.workspace_status(ws) == 0
    buf = ws.cpu().numpy()
    toff, tpoints = single_pass_table(L)
    words = np.frombuffer(buf[toff:toff + tpoints * 64].tobytes(), dtype=np.uint32).reshape(4, tpoints, 4)
    sk = oracle.words_to_int(pr["sk"])
    R = [[oracle.words_to_int(pr["r"][c, j]) for j in range(l)] for c in range(n)]
    Bm = pr["B"].astype(np.int64)
    A64 = A_h.astype(np.int64)
    mask = (1 << w) - 1
    checked = 0
    for s in range(L["nstrips"]):
        cols = list(range(s * k, min(s * k + k, n)))
        codes = np.zeros(m, dtype=np.int64)
        for t, c in enumerate(cols):
            codes |= A64[:, c] << (w * t)
        distinct = [int(u) for u in np.unique(codes[codes != 0])]
        scal, idx = [], []
        for e, u in enumerate(distinct):
            parts = [((u >> (w * t)) & mask, col) for t, col in enumerate(cols)]
            for j in range(l):
                s1 = sum(ut * R[col][j] for ut, col in parts) % Q
                s2 = sum(ut * (R[col][j] * sk + int(Bm[col, j])) for ut, col in parts) % Q
                for c, sc in ((0, s1), (1, s2)):
                    scal.append(sc)
                    idx.append(((s * L["emax"] + e) * 2 + c) * L["lp"] + j)
        sw = np.frombuffer(b"".join(int(x).to_bytes(32, "little") for x in scal), dtype="<u4").reshape(-1, 8)
        want = oracle.base_mul_comb(sw)
        idx = np.asarray(idx)
        got = np.concatenate([words[q, idx] for q in range(4)], axis=1)
        assert np.array_equal(got, want), s
        checked += len(idx)
    assert checked > 0
