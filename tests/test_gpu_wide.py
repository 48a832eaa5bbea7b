"""GPU parity of the wide-value path (plaintext entries of up to 16 bits,
the paper's t = 12 and 16 grid) against the CPU oracle, bit-exact: ragged
multi-tile shapes, columns of repeated and extreme values, more rows than
2^11 (long level-1 lists), crafted exceptional additions, the device status
word for out-of-range entries, and sampled parity at 1024 x 1024 x 256."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import Q, device, encrypt_gpu, mismatches, run_affine

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    return device()


def _problem(dev, seed, m, n, l, w):
    pr = inputs.pcmm_problem(seed, m, n, l, w)
    ctB = encrypt_gpu(dev, pr)
    return pr, pcmm.plaintext16(pr["A"], dev), ctB


def _want(A, pr):
    return oracle.closed_form(A, pr["r"], pr["sk"], pr["B"]).reshape(-1, 2, 16)


@pytest.mark.parametrize("w", [9, 12, 16])
def test_wide_ragged_multi_tile_shapes(dev, w):
    m, n, l = 70, 37, 45
    pr, A, ctB = _problem(dev, 1500 + w, m, n, l, w)
    want = _want(pr["A"], pr)
    for k in (1, 0):
        got = run_affine(lambda: pcmm.cussen16(A, ctB, l, w, k=k), m * l)
        assert mismatches(got, want) == 0, (w, k)
    got = run_affine(lambda: pcmm.schoolbook16(A, ctB, l, w), m * l)
    assert mismatches(got, want) == 0


def test_wide_duplicates_and_extremes(dev):
    # Columns drawn from {0, 1, 2, 2^15, 2^16 - 2, 2^16 - 1} (many duplicates,
    # both ends of the range), one column of distinct values, one of zeros.
    m, n, l, w = 64, 7, 33, 16
    pr = inputs.pcmm_problem(1600, m, n, l, 8)
    rng = np.random.default_rng(1601)
    Ah = rng.choice(np.array([0, 1, 2, 0x8000, 0xFFFE, 0xFFFF], dtype=np.uint16), size=(m, n))
    Ah[:, 3] = np.arange(m, dtype=np.uint16) * 1021 + 7
    Ah[:, 5] = 0
    ctB = encrypt_gpu(dev, pr)
    A = pcmm.plaintext16(Ah, dev)
    want = _want(Ah, pr)
    got = run_affine(lambda: pcmm.cussen16(A, ctB, l, w, k=1), m * l)
    assert mismatches(got, want) == 0
    got = run_affine(lambda: pcmm.schoolbook16(A, ctB, l, w), m * l)
    assert mismatches(got, want) == 0


def test_wide_many_rows(dev):
    # 3000 rows of 16-bit values: about 2930 distinct values per column, so
    # level-1 lists and ranks go well past 2^11 entries.
    m, n, l, w = 3000, 3, 8, 16
    pr, A, ctB = _problem(dev, 1700, m, n, l, w)
    ws = pcmm.workspace(m, n, l, w, 1, device=dev)
    jac = pcmm.cussen16(A, ctB, l, w, k=1, ws=ws)
    aff = pcmm.normalize(jac, m * l)
    torch.cuda.synchronize()
    assert pcmm.workspace_status(ws) == 0
    got = pcmm.planar_to_ct(pcmm.to_host_words(aff), m * l)
    want = _want(pr["A"], pr)
    assert mismatches(got, want) == 0


@pytest.mark.parametrize("mode,m,w", [("equal", 12, 12), ("cancel", 12, 12), ("infinity", 12, 12),
                                      ("infinity", 80, 16), ("equal", 80, 16)])
def test_wide_exceptional_additions(dev, mode, m, w):
    # Enc(B) replaced by points u G of chosen discrete logs so that equal
    # points, opposite points and infinity meet inside the table build and
    # the gather; the expected product is (sum_k a_ik u_kj) G.  With 80
    # rows of 16-bit values level 2 is long enough to be built as a chain
    # over an affine level 3, and infinity inputs send it down its fallback.
    n, l = 6, 3
    rng = np.random.default_rng(1800)
    Ah = rng.integers(0, 1 << w, size=(m, n), dtype=np.uint16)
    Ah[:, 0] = np.arange(m, dtype=np.uint16) * 3        # an arithmetic column: equal differences
    u = np.zeros((n, l, 2), dtype=object)
    for k in range(n):
        for j in range(l):
            for c in range(2):
                if mode == "equal":
                    u[k, j, c] = 1 + c
                elif mode == "cancel":
                    u[k, j, c] = (5 + j) if k % 2 == 0 else Q - (5 + j)
                else:
                    u[k, j, c] = 0 if (k + j + c) % 3 == 0 else 3 + k
    if mode == "cancel":
        Ah[:, 1::2] = Ah[:, 0::2][:, : Ah[:, 1::2].shape[1]]
    pts = oracle.base_mul(np.stack([oracle.int_to_words(int(v)) for v in u.ravel()])).reshape(n, l, 2, 16)
    want_s = [sum(int(Ah[i, k]) * int(u[k, j, c]) for k in range(n)) % Q
              for i in range(m) for j in range(l) for c in range(2)]
    want = oracle.base_mul(np.stack([oracle.int_to_words(v) for v in want_s])).reshape(m * l, 2, 16)
    ctB = pcmm.to_device_words(pcmm.ct_to_planar(pts), dev)
    A = pcmm.plaintext16(Ah, dev)
    assert mismatches(run_affine(lambda: pcmm.cussen16(A, ctB, l, w, k=1), m * l), want) == 0
    assert mismatches(run_affine(lambda: pcmm.schoolbook16(A, ctB, l, w), m * l), want) == 0


def test_wide_out_of_range_entries_raise_status(dev):
    m, n, l, w = 8, 6, 4, 12
    pr, A, ctB = _problem(dev, 1900, m, n, l, w)
    Ah = pr["A"].copy()
    Ah[3, 2] = 1 << w
    A2 = pcmm.plaintext16(Ah, dev)
    ws = pcmm.workspace(m, n, l, w, 1, device=dev)
    pcmm.cussen16(A2, ctB, l, w, k=1, ws=ws)
    assert pcmm.workspace_status(ws) & 1
    pcmm.cussen16(A, ctB, l, w, k=1, ws=ws)
    assert pcmm.workspace_status(ws) == 0
    with pytest.raises(pcmm.PcmmError) as ei:
        pcmm.cussen16(A, ctB, l, 17, k=1, ws=ws)
    assert ei.value.status == 1
    with pytest.raises(TypeError):
        pcmm.cussen16(torch.zeros((m, n), dtype=torch.uint8, device=dev), ctB, l, w)


@pytest.mark.parametrize("w", [12, 16])
def test_wide_full_size_sampled(dev, w):
    m, n, l = 1024, 1024, 256
    pr, A, ctB = _problem(dev, inputs.SEED_BASE + 2, m, n, l, w)
    k = pcmm.choose_k(m, n, l, w)
    assert k == 1
    ws = pcmm.workspace(m, n, l, w, k, device=dev)
    jac = pcmm.cussen16(A, ctB, l, w, k=k, ws=ws)
    aff = pcmm.normalize(jac, m * l)
    torch.cuda.synchronize()
    assert pcmm.workspace_status(ws) == 0
    got = pcmm.planar_to_ct(pcmm.to_host_words(aff), m * l)
    rng = np.random.default_rng(w)
    pairs = np.stack([rng.integers(0, m, 64), rng.integers(0, l, 64)], axis=1)
    pairs = np.concatenate([pairs, [[0, 0], [m - 1, l - 1]]])
    want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"], pairs=pairs)
    assert mismatches(got[pairs[:, 0] * l + pairs[:, 1]], want) == 0


def test_wide_maximum_rows(dev):
    # 70000 rows of 16-bit values: about 43000 distinct values per column, so
    # the level-1 lists, tracking pointers, ranks and strip tables run close
    # to the 2^16 - 1 entries the 16-bit plan arrays allow.
    m, n, l, w = 70000, 2, 1, 16
    pr, A, ctB = _problem(dev, 2000, m, n, l, w)
    ws = pcmm.workspace(m, n, l, w, 1, device=dev)
    jac = pcmm.cussen16(A, ctB, l, w, k=1, ws=ws)
    aff = pcmm.normalize(jac, m * l)
    torch.cuda.synchronize()
    assert pcmm.workspace_status(ws) == 0
    got = pcmm.planar_to_ct(pcmm.to_host_words(aff), m * l)
    rng = np.random.default_rng(2001)
    rows = np.concatenate([rng.integers(0, m, 120), [0, m - 1]])
    # Rows holding the smallest and largest values of each column too.
    for c in range(n):
        rows = np.concatenate([rows, [int(np.argmin(pr["A"][:, c])), int(np.argmax(pr["A"][:, c]))]])
    pairs = np.stack([rows, np.zeros_like(rows)], axis=1)
    want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"], pairs=pairs)
    assert mismatches(got[rows], want) == 0


@pytest.mark.parametrize("w", [4, 16])
def test_vector_times_ciphertext_scalars(dev, w):
    # The paper's plaintext-vector x ciphertext-scalar product: A is one
    # column (n = 1), Enc(B) a row of independent scalars, as bench.py's
    # vector workload runs it.
    m, n, l = 512, 1, 200
    pr = inputs.pcmm_problem(2100 + w, m, n, l, w)
    ctB = encrypt_gpu(dev, pr)
    A = pcmm.plaintext16(pr["A"], dev) if w > 8 else torch.from_numpy(pr["A"]).to(dev)
    for fn in (lambda: pcmm.cussen(A, ctB, l, w, k=1), lambda: pcmm.schoolbook(A, ctB, l, w)):
        got = run_affine(fn, m * l)
        rng = np.random.default_rng(w)
        pairs = np.stack([rng.integers(0, m, 80), rng.integers(0, l, 80)], axis=1)
        pairs = np.concatenate([pairs, [[0, 0], [m - 1, l - 1]]])
        want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"], pairs=pairs)
        assert mismatches(got[pairs[:, 0] * l + pairs[:, 1]], want) == 0
