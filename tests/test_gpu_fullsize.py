"""Parity of EVERY output at the benchmark's own sizes (Algorithm 3 loses
no accuracy: each output ciphertext must equal the closed form
C1_ij = (sum_k a_ik r_kj) G, C2_ij = (sum_k a_ik (r_kj x + b_kj)) G of
Eq. ahe_5_elgamal with H = x G, bit for bit after affine normalisation).

These take a few minutes of host time for the oracle (all cores), so they
carry the ``slow`` mark besides ``gpu``."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import device, encrypt_gpu, mismatches

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    return device()


def _affine_host(jac, count):
    aff = pcmm.normalize(jac, count)
    torch.cuda.synchronize()
    return pcmm.planar_to_ct(pcmm.to_host_words(aff), count)


@pytest.mark.parametrize("w,k", [(8, 1), (4, 2), (16, 1)])
def test_headline_product_every_output(dev, w, k):
    """1024 x 1024 times Enc(1024 x 256) in the benchmark's configuration
    (default workspace: two passes of strips at w = 8, k = 1; one wave per
    pass at the paper's w = 16): all 262,144 output ciphertexts (524,288
    points) against the closed form."""
    m, n, l = 1024, 1024, 256
    pr = inputs.pcmm_problem(inputs.SEED_BASE + 2, m, n, l, w)
    ctB = encrypt_gpu(dev, pr)
    A = pcmm.plaintext16(pr["A"], dev) if w > 8 else torch.from_numpy(pr["A"]).to(dev)
    ws = pcmm.workspace(m, n, l, w, k, device=dev)
    got = _affine_host(pcmm.cussen(A, ctB, l, w, k=k, ws=ws), m * l)
    assert pcmm.workspace_status(ws) == 0
    want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"]).reshape(m * l, 2, 16)
    assert mismatches(got, want) == 0


def test_batched_workload_every_output_of_every_instance(dev):
    """The 64-instance batched workload (m, n, l uniform in [32, 768], w in
    1..8, cost-model k) in one persistent launch; every output of every
    instance against the closed form: 9,816,999 output ciphertexts."""
    shapes = inputs.batched_shapes(inputs.SEED_BASE + 4, count=64)
    items, probs = [], []
    for i, (m, n, l, w) in enumerate(shapes):
        pr = inputs.pcmm_problem(5200 + i, m, n, l, w)
        items.append((torch.from_numpy(pr["A"]).to(dev), encrypt_gpu(dev, pr), l, w, 0))
        probs.append(pr)
    b = pcmm.Batch(items)
    outs = b.run()
    torch.cuda.synchronize()
    assert pcmm.workspace_status(b.ws) == 0
    compared = 0
    for (m, n, l, w), pr, out in zip(shapes, probs, outs):
        got = _affine_host(out, m * l)
        want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"]).reshape(m * l, 2, 16)
        assert mismatches(got, want) == 0, (m, n, l, w)
        compared += m * l
    assert compared == 9816999


def test_sweep_point_every_output(dev):
    """One square sweep point in full: 512 x 512 times Enc(512 x 512), w = 5
    (cost-model k = 1, one pass), all 262,144 outputs against the closed form."""
    n, w = 512, 5
    seed = inputs.SEED_BASE + 3
    pr = inputs.pcmm_problem(seed, n, n, n, 1)
    Ah = inputs.plaintext_matrix(seed, n, n, w)
    ctB = encrypt_gpu(dev, pr)
    A = torch.from_numpy(Ah).to(dev)
    k = pcmm.choose_k(n, n, n, w)
    ws = pcmm.workspace(n, n, n, w, k, device=dev)
    got = _affine_host(pcmm.cussen(A, ctB, n, w, k=k, ws=ws), n * n)
    assert pcmm.workspace_status(ws) == 0
    want = oracle.closed_form(Ah, pr["r"], pr["sk"], pr["B"]).reshape(n * n, 2, 16)
    assert mismatches(got, want) == 0


def _lines(n, extra=()):
    """Output indices (i, j) of rows 0 and n - 1, columns 0 and n - 1, and
    of the rows and columns listed in extra, each counted once."""
    sel = np.zeros((n, n), dtype=bool)
    for t in (0, n - 1) + tuple(extra):
        sel[t, :] = True
        sel[:, t] = True
    ii, jj = np.nonzero(sel)
    return np.stack([ii, jj], axis=1)


@pytest.mark.parametrize("n,w", [(512, 5), (2048, 7), (2048, 1), (1024, 8)])
def test_sweep_rows_and_columns(dev, n, w):
    """The square sweep (A n x n, Enc(B) n x n) as bench.py runs it
    (cost-model k, default workspace; several strip passes at n = 2048):
    every output of rows and columns 0, 31, 32, 127, 128 and n - 1 (the
    first and last rows and columns, the 32-column warp boundary, the
    128-thread block boundary of the gather rows) against the closed form:
    12 n - 36 outputs per size (6108 at n = 512, 24540 at n = 2048)."""
    seed = inputs.SEED_BASE + 3
    pr = inputs.pcmm_problem(seed, n, n, n, 1)
    Ah = inputs.plaintext_matrix(seed, n, n, w)
    ctB = encrypt_gpu(dev, pr)
    A = torch.from_numpy(Ah).to(dev)
    k = pcmm.choose_k(n, n, n, w)
    ws = pcmm.workspace(n, n, n, w, k, device=dev)
    got = _affine_host(pcmm.cussen(A, ctB, n, w, k=k, ws=ws), n * n)
    assert pcmm.workspace_status(ws) == 0
    pairs = _lines(n, extra=(31, 32, 127, 128))
    assert len(pairs) == 12 * n - 36
    want = oracle.closed_form(Ah, pr["r"], pr["sk"], pr["B"], pairs=pairs)
    assert mismatches(got[pairs[:, 0] * n + pairs[:, 1]], want) == 0
