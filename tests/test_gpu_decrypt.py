"""GPU decryption (Section 2.4: m = log_G(C2 - x C1) in [0, mmax] by
baby-step giant-step) against the messages the ciphertexts were built from
and against the CPU oracle's decryption: edge messages around every
boundary of the search (0, multiples of the baby-step count, mmax, mmax + 1,
"negative" messages, ciphertexts with C1 at infinity), several baby-step
counts, the baby-step table read back slot by slot, a wrong key, and the
full 1024 x 1024 x 256 PC-MM output decrypted to the integer product A B."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import Q, ct_from_aos, device, encrypt_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    return device()


def _craft(sk: int, items):
    """Ciphertexts (r G, r H + v G) for (r, v) pairs (r = 0: C1 at infinity),
    built by the oracle: [count, 2, 16]."""
    G = oracle.generator()
    H = oracle.keygen(sk)
    out = np.zeros((len(items), 2, 16), dtype=np.uint32)
    for i, (r, v) in enumerate(items):
        c1 = oracle.scalar_mul(r % Q, G)
        c2 = oracle.point_add(oracle.scalar_mul(r % Q, H), oracle.scalar_mul(v % Q, G))
        out[i, 0], out[i, 1] = c1, c2
    return out


def _decrypt(dev, sk_words, ct_aos, mmax, steps):
    ct = ct_from_aos(dev, ct_aos)
    out = pcmm.decrypt(sk_words, ct, ct_aos.shape[0], mmax, steps)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _edge_items(rng, mmax, baby):
    vs = [0, 1, 2, 3, baby - 1, baby, baby + 1, 2 * baby, mmax - 1, mmax, mmax + 1,
          mmax + baby, (mmax // baby) * baby, (mmax // baby + 1) * baby - 1, 2 * mmax + 7,
          Q - 1, Q - baby, Q - mmax, 2**200 + 5]
    vs += [int(x) for x in rng.integers(0, mmax + 1, 45)]
    items = [(int.from_bytes(rng.bytes(32), "little") % (Q - 1) + 1, v) for v in vs]
    items += [(0, 0), (0, 77 % (mmax + 1)), (0, mmax + 5), (1, 0), (Q - 1, 3)]
    return items


@pytest.mark.parametrize("baby", [0, 64, 7, 1])
def test_decrypt_edge_messages(dev, baby):
    # baby = 0: the library's default for the range (one giant step here).
    rng = np.random.default_rng(11 + baby)
    sk = int.from_bytes(rng.bytes(32), "little") % (Q - 1) + 1
    mmax = 700 if baby == 1 else 5000
    steps = pcmm.BabySteps(baby, device=dev) if baby else pcmm.BabySteps.for_range(mmax, device=dev)
    items = _edge_items(rng, mmax, steps.baby)
    ct = _craft(sk, items)
    want = np.array([v % Q if v % Q <= mmax else -1 for _, v in items], dtype=np.int64)
    got = _decrypt(dev, oracle.int_to_words(sk), ct, mmax, steps)
    assert (got == want).all(), np.nonzero(got != want)
    assert (oracle.decrypt(sk, ct, mmax) == want).all()


def test_decrypt_encrypted_bytes_ragged(dev):
    # Every byte value, a count that is not a multiple of the warp size.
    pr = {"B": np.arange(300, dtype=np.int64).astype(np.uint8)}
    s = inputs.streams(5)
    pr["sk"] = inputs.uniform_scalars(s["sk"], (1,))[0]
    pr["r"] = inputs.uniform_scalars(s["r"], (300,))
    ct = encrypt_gpu(dev, pr)
    steps = pcmm.BabySteps.for_range(255, device=dev)
    out = pcmm.decrypt(pr["sk"], ct, 300, 255, steps)
    assert (out.cpu().numpy() == pr["B"].astype(np.int64)).all()
    # A narrower range: messages above it report -1.
    out = pcmm.decrypt(pr["sk"], ct, 300, 99, steps)
    want = np.where(pr["B"] <= 99, pr["B"].astype(np.int64), -1)
    assert (out.cpu().numpy() == want).all()
    # The degenerate range [0, 0] (its own table: 32 baby steps), and an
    # empty call, which launches nothing.
    zero = pcmm.BabySteps.for_range(0, device=dev)
    out = pcmm.decrypt(pr["sk"], ct, 300, 0, zero)
    assert (out.cpu().numpy() == np.where(pr["B"] == 0, 0, -1)).all()
    empty = torch.full((4,), 7, dtype=torch.int64, device=dev)
    pcmm.decrypt(pr["sk"], ct, 0, 255, steps, out=empty)
    assert (empty.cpu().numpy() == 7).all()


def test_wrong_key_finds_nothing(dev):
    pr = inputs.pcmm_problem(inputs.SEED_BASE + 7, 4, 4, 64, 8)
    ct = encrypt_gpu(dev, {"B": pr["B"], "sk": pr["sk"], "r": pr["r"]})
    wrong = oracle.int_to_words((oracle.words_to_int(pr["sk"]) + 1) % Q)
    steps = pcmm.BabySteps.for_range(255, device=dev)
    out = pcmm.decrypt(wrong, ct, 4 * 64, 255, steps).cpu().numpy()
    # M = C2 - (x + 1) C1 = b G - C1: in [0, 255] G only with negligible probability.
    assert (out == -1).all()


def test_baby_step_table_slots(dev):
    # Every slot holds (word 1 of x(j G), j + 1) for a distinct j in
    # [1, baby), reachable by linear probing from word 0 of x(j G).
    baby = 1000
    steps = pcmm.BabySteps(baby, device=dev)
    torch.cuda.synchronize()
    slots = steps.table.cpu().numpy().view(np.uint64)
    cap = slots.size
    assert cap == 2048
    pts = oracle.base_mul(np.stack([oracle.int_to_words(j) for j in range(1, baby)]))
    want = {(int(p[1]), j + 1): int(p[0]) for j, p in zip(range(1, baby), pts)}
    full = np.nonzero(slots)[0]
    assert full.size == baby - 1
    seen = set()
    for pos in full:
        e = int(slots[pos])
        key = (e >> 32, e & 0xFFFFFFFF)
        assert key in want, key
        home = want[key] & (cap - 1)
        d = (int(pos) - home) % cap
        assert all(slots[(home + t) % cap] != 0 for t in range(d + 1))
        seen.add(key)
    assert len(seen) == baby - 1


def test_full_size_pcmm_output_decrypts_to_product(dev):
    # The benchmark's w = 8 product, every output decrypted on the GPU and
    # compared with the integer product A B.
    m, n, l, w = 1024, 1024, 256, 8
    pr = inputs.pcmm_problem(inputs.SEED_BASE + 2, m, n, l, w)
    ctB = encrypt_gpu(dev, pr)
    A = torch.from_numpy(pr["A"]).to(dev)
    jac = pcmm.cussen(A, ctB, l, w)
    ct = pcmm.normalize(jac, m * l)
    del jac
    mmax = n * (2**w - 1) * 255
    steps = pcmm.BabySteps.for_range(mmax, device=dev)
    assert steps.baby == 1 << 24
    got = pcmm.decrypt(pr["sk"], ct, m * l, mmax, steps).cpu().numpy().reshape(m, l)
    AB = pr["A"].astype(np.int64) @ pr["B"].astype(np.int64)
    assert (got == AB).all()
    # Half the range: entries above it report -1, the rest are unchanged.
    half = mmax // 2
    got = pcmm.decrypt(pr["sk"], ct, m * l, half, steps).cpu().numpy().reshape(m, l)
    assert (got == np.where(AB <= half, AB, -1)).all()
