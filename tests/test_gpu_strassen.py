"""GPU Strassen PC-MM (Section 3.1; pcmm_strassen) against the CPU oracle,
bit-exact after affine normalisation: every output of small and medium
shapes at every recursion depth against the closed form, crafted inputs
whose block sums are negative, zero or cancel, the oracle's own Strassen
recursion, out-of-range plaintext flags and argument errors."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import ct_from_aos, device, encrypt_gpu, mismatches, run_affine

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    return device()


def _problem(dev, seed, m, n, l, w):
    pr = inputs.pcmm_problem(seed, m, n, l, w)
    return pr, torch.from_numpy(pr["A"]).to(dev), encrypt_gpu(dev, pr)


def _want(pr):
    return oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"]).reshape(-1, 2, 16)


@pytest.mark.parametrize("m,n,l,w", [(8, 8, 8, 4), (16, 32, 24, 8), (32, 16, 64, 1), (64, 64, 40, 5)])
def test_every_depth_matches_closed_form(dev, m, n, l, w):
    """Every output (m l ciphertexts) at each depth the shape allows."""
    pr, A, ctB = _problem(dev, 9100 + m + n + l + w, m, n, l, w)
    want = _want(pr)
    d = 0
    while d <= 4 and m % (1 << d) == 0 and n % (1 << d) == 0 and l % (1 << d) == 0:
        ws = torch.empty(pcmm.strassen_workspace_bytes(m, n, l, w, d), dtype=torch.uint8, device=dev)
        got = run_affine(lambda: pcmm.strassen(A, ctB, l, w, d, ws=ws), m * l)
        assert pcmm.workspace_status(ws) == 0
        assert mismatches(got, want) == 0, d
        d += 1


def test_medium_shape_every_output(dev):
    """256 x 256 times Enc(256 x 256), w = 8, three levels (343 leaves of
    32 x 32 blocks): all 65,536 outputs against the closed form."""
    m = n = l = 256
    pr, A, ctB = _problem(dev, 9200, m, n, l, 8)
    got = run_affine(lambda: pcmm.strassen(A, ctB, l, 8, 3), m * l)
    assert mismatches(got, _want(pr)) == 0


def test_negative_zero_and_cancelling_block_sums(dev):
    """A21 = A11 + 1 and A12 = A22 (block differences of both signs and
    zero), B12 = B22 and B21 = -B11 (ciphertext sums at infinity): against
    the oracle's schoolbook and its Strassen recursion."""
    m = n = l = 8
    pr = inputs.pcmm_problem(777, m, n, l, 4)
    A = pr["A"].astype(np.int64)
    A[4:, :4] = np.minimum(A[:4, :4] + 1, 15)
    A[:4, 4:] = A[4:, 4:]
    A = A.astype(np.uint8)
    r, B = pr["r"].copy(), pr["B"].copy()
    r[:4, 4:] = r[4:, 4:]
    B[:4, 4:] = B[4:, 4:]
    ct = oracle.encrypt(oracle.keygen(pr["sk"]), B, r)
    for k in range(4):
        for j in range(4):
            for c in range(2):
                ct[4 + k, j, c] = oracle.point_neg(ct[k, j, c])
    want, _ = oracle.schoolbook(A, ct, 4)
    want = want.reshape(-1, 2, 16)
    Ad, ctd = torch.from_numpy(A).to(dev), ct_from_aos(dev, ct)
    for d in (1, 2, 3):
        got = run_affine(lambda: pcmm.strassen(Ad, ctd, l, 4, d), m * l)
        assert mismatches(got, want) == 0, d
        ora, _ = oracle.strassen(A, ct, 4, d)
        assert mismatches(got, ora.reshape(-1, 2, 16)) == 0, d


def test_out_of_range_entries_and_errors(dev):
    m, n, l, w = 16, 16, 8, 3
    pr, A, ctB = _problem(dev, 9300, m, n, l, w)
    for d in (0, 2):
        ws = torch.empty(pcmm.strassen_workspace_bytes(m, n, l, w, d), dtype=torch.uint8, device=dev)
        A2 = A.clone()
        A2[5, 9] = 200
        pcmm.strassen(A2, ctB, l, w, d, ws=ws)
        assert pcmm.workspace_status(ws) & 1
        got = run_affine(lambda: pcmm.strassen(A, ctB, l, w, d, ws=ws), m * l)
        assert pcmm.workspace_status(ws) == 0
        assert mismatches(got, _want(pr)) == 0
    small = torch.empty(512, dtype=torch.uint8, device=dev)
    with pytest.raises(pcmm.PcmmError) as e:
        pcmm.strassen(A, ctB, l, w, 2, ws=small)
    assert e.value.status == 2
    with pytest.raises(pcmm.PcmmError) as e:
        pcmm.strassen(A, ctB, l, w, 4, ws=small)          # l = 8 not a multiple of 16
    assert e.value.status == 1


@pytest.mark.parametrize("w", [12, 16])
def test_wide_entries_every_depth(dev, w):
    """pcmm_strassen16 (the paper's t = 12 and 16): every output at depths
    0..4 of 32 x 32 times Enc(32 x 32); the block sums are int16 while
    w + depth <= 15 and int32 beyond, so both layouts are exercised."""
    m = n = l = 32
    pr = inputs.pcmm_problem(9400 + w, m, n, l, 1)
    Ah = inputs.plaintext_matrix(9400 + w, m, n, w)
    A = pcmm.plaintext16(Ah, dev)
    ctB = encrypt_gpu(dev, pr)
    want = oracle.closed_form(Ah, pr["r"], pr["sk"], pr["B"]).reshape(-1, 2, 16)
    for d in range(5):
        got = run_affine(lambda: pcmm.strassen(A, ctB, l, w, d), m * l)
        assert mismatches(got, want) == 0, d
    ora, _ = oracle.strassen(Ah, oracle.encrypt(oracle.keygen(pr["sk"]), pr["B"], pr["r"]), w, 2)
    assert mismatches(run_affine(lambda: pcmm.strassen(A, ctB, l, w, 2), m * l), ora.reshape(-1, 2, 16)) == 0


def test_deepest_recursion_to_single_entries(dev):
    """Depth 7 on 128 x 128 times Enc(128 x 128): recursion down to 1 x 1
    blocks (823,543 leaves, as in the paper's count model), every one of the
    16,384 outputs against the closed form; w = 8 at depth 7 is the widest
    int16 case (|block sums| <= 2^7 255)."""
    m = n = l = 128
    for w in (1, 8):
        pr, A, ctB = _problem(dev, 9500 + w, m, n, l, w)
        got = run_affine(lambda: pcmm.strassen(A, ctB, l, w, 7), m * l)
        assert mismatches(got, _want(pr)) == 0, w
