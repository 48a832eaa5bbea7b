"""GPU parity of encryption and of the PC-MM path (schoolbook, Cussen for
every strip width, normalisation) against the CPU oracle, element by
element and bit-exact: tiny and ragged multi-tile shapes, every bit-width,
degenerate shapes, crafted exceptional additions, infinity inputs, chunked
passes, device status reporting and argument errors; plus sampled parity at
the full 1024 x 1024 x 256 size in the configuration the benchmark times."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import Q, ct_from_aos, device, encrypt_gpu, mismatches, run_affine

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    return device()


def test_encrypt_matches_oracle(dev):
    # Every message byte, a ragged count (not a multiple of the warp size).
    s = inputs.streams(99)
    sk = inputs.uniform_scalars(s["sk"], (1,))[0]
    H = oracle.keygen(sk)
    msg = np.arange(1000, dtype=np.int64).astype(np.uint8)
    r = inputs.uniform_scalars(s["r"], (1000,))
    r[0] = oracle.int_to_words(1)
    r[1] = oracle.int_to_words(Q - 1)
    r[2] = oracle.int_to_words(2**248)           # single non-zero top window
    pr = {"sk": sk, "B": msg, "r": r}
    ct = encrypt_gpu(dev, pr, H)
    torch.cuda.synchronize()
    got = pcmm.planar_to_ct(pcmm.to_host_words(ct), 1000)
    want = oracle.encrypt(H, msg, r)
    assert mismatches(got, want) == 0


def _problem(dev, seed, m, n, l, w, msg_bits=8):
    pr = inputs.pcmm_problem(seed, m, n, l, w, msg_bits)
    ctB = encrypt_gpu(dev, pr)
    A = torch.from_numpy(pr["A"]).to(dev)
    return pr, A, ctB


def _want(pr):
    return oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"]).reshape(-1, 2, 16)


def test_tiny_config_all_methods(dev):
    m = n = l = 16
    pr, A, ctB = _problem(dev, inputs.SEED_BASE + 1, m, n, l, 4, msg_bits=4)
    want = _want(pr)
    assert mismatches(run_affine(lambda: pcmm.schoolbook(A, ctB, l, 4), m * l), want) == 0
    for k in (1, 2, 3, 0):
        got = run_affine(lambda: pcmm.cussen(A, ctB, l, 4, k=k), m * l)
        assert mismatches(got, want) == 0, k
    dec = oracle.decrypt(pr["sk"], got.reshape(m, l, 2, 16), n * 15 * 15)
    assert (dec == pr["A"].astype(np.int64) @ pr["B"].astype(np.int64)).all()


@pytest.mark.parametrize("w", [1, 2, 4, 8])
def test_ragged_multi_tile_shapes(dev, w):
    # l = 45 spans two 32-column warps with a ragged tail; n = 37 leaves a
    # ragged last strip for k > 1; m = 70 spans several warps of rows.
    m, n, l = 70, 37, 45
    pr, A, ctB = _problem(dev, 500 + w, m, n, l, w)
    want = _want(pr)
    ks = sorted({1, 2, 12 // w, 16 // w, 0} - {k for k in (2, 12 // w, 16 // w) if w * k > 16})
    for k in ks:
        got = run_affine(lambda: pcmm.cussen(A, ctB, l, w, k=k), m * l)
        assert mismatches(got, want) == 0, (w, k)
    if w in (1, 8):
        got = run_affine(lambda: pcmm.schoolbook(A, ctB, l, w), m * l)
        assert mismatches(got, want) == 0


def test_degenerate_shapes(dev):
    for (m, n, l, w) in [(1, 1, 1, 4), (1, 5, 1, 8), (3, 1, 33, 2), (40, 3, 1, 3)]:
        pr, A, ctB = _problem(dev, 600 + m + n + l, m, n, l, w)
        want = _want(pr)
        for k in (1, 0):
            assert mismatches(run_affine(lambda: pcmm.cussen(A, ctB, l, w, k=k), m * l), want) == 0
        assert mismatches(run_affine(lambda: pcmm.schoolbook(A, ctB, l, w), m * l), want) == 0


def test_zero_matrix_and_zero_rows(dev):
    m, n, l, w = 9, 6, 5, 4
    pr, A, ctB = _problem(dev, 700, m, n, l, w)
    Ah = pr["A"].copy()
    Ah[2] = 0
    Ah[:, 4] = 0
    pr2 = dict(pr, A=Ah)
    want = _want(pr2)
    A2 = torch.from_numpy(Ah).to(dev)
    for k in (1, 2, 3):
        assert mismatches(run_affine(lambda: pcmm.cussen(A2, ctB, l, w, k=k), m * l), want) == 0
    Z = torch.zeros_like(A)
    got = run_affine(lambda: pcmm.cussen(Z, ctB, l, w, k=1), m * l)
    assert not got.any()
    got = run_affine(lambda: pcmm.schoolbook(Z, ctB, l, w), m * l)
    assert not got.any()


@pytest.mark.parametrize("density,w", [(0.02, 8), (0.2, 4), (0.005, 1)])
def test_sparse_plaintext(dev, density, w):
    # Pruned-weight style A: most entries zero, whole zero strips for k > 1
    # and rows with no non-zero entry at all.  Every output against the
    # closed form, for k = 1, the cost-model k and a wide strip.
    m, n, l = 150, 301, 70
    pr = inputs.pcmm_problem(820 + w, m, n, l, w)
    pr["A"] = inputs.sparse_plaintext(820 + w, m, n, w, density)
    pr["A"][3] = 0
    ctB = encrypt_gpu(dev, pr)
    A = torch.from_numpy(pr["A"]).to(dev)
    want = _want(pr)
    for k in sorted({1, pcmm.choose_k(m, n, l, w), 16 // w if w > 1 else 8}):
        got = run_affine(lambda: pcmm.cussen(A, ctB, l, w, k=k), m * l)
        assert mismatches(got, want) == 0, k
    assert not got.reshape(m, l, 2, 16)[3].any()


def _crafted(seed, m, n, l, w, mode):
    """Enc(B) replaced by points u G of chosen discrete logs; the expected
    product (sum_k a_ik u_kj) G is computed by the oracle from the scalars."""
    rng = np.random.default_rng(seed)
    A = rng.integers(0, 2**w, size=(m, n), dtype=np.uint8)
    u = np.zeros((n, l, 2), dtype=object)
    for k in range(n):
        for j in range(l):
            for c in range(2):
                if mode == "equal":
                    u[k, j, c] = 1 + c
                elif mode == "cancel":
                    u[k, j, c] = (5 + j) if k % 2 == 0 else Q - (5 + j)
                elif mode == "infinity":
                    u[k, j, c] = 0 if (k + j + c) % 3 == 0 else 3 + k
                else:
                    u[k, j, c] = int(rng.integers(1, 2**20))
    if mode == "cancel":
        A[:, 1::2] = A[:, 0::2][:, : A[:, 1::2].shape[1]]
    pts = oracle.base_mul(np.stack([oracle.int_to_words(int(v)) for v in u.ravel()])).reshape(n, l, 2, 16)
    want_s = np.zeros((m, l, 2), dtype=object)
    for i in range(m):
        for j in range(l):
            for c in range(2):
                want_s[i, j, c] = sum(int(A[i, k]) * int(u[k, j, c]) for k in range(n)) % Q
    want = oracle.base_mul(np.stack([oracle.int_to_words(int(v)) for v in want_s.ravel()]))
    return A, pts, want.reshape(m * l, 2, 16)


@pytest.mark.parametrize("mode", ["equal", "cancel", "infinity", "small"])
def test_exceptional_additions(dev, mode):
    m, n, l, w = 12, 8, 35, 3
    A, pts, want = _crafted(31, m, n, l, w, mode)
    Ad = torch.from_numpy(A).to(dev)
    ctB = ct_from_aos(dev, pts)
    for k in (1, 2, 4):
        assert mismatches(run_affine(lambda: pcmm.cussen(Ad, ctB, l, w, k=k), m * l), want) == 0, k
    assert mismatches(run_affine(lambda: pcmm.schoolbook(Ad, ctB, l, w), m * l), want) == 0


def test_chunked_passes_match_single_pass(dev):
    m, n, l, w = 40, 29, 40, 4
    pr, A, ctB = _problem(dev, 800, m, n, l, w)
    want = _want(pr)
    passes = 0
    for k in (1, 2):
        full = pcmm.cussen_workspace_bytes(m, n, l, w, k)
        # Smaller workspaces hold fewer strips and force several passes.
        for nb in (full, full // 3, full // 8):
            ws = torch.empty(nb, dtype=torch.uint8, device=dev)
            try:
                got = run_affine(lambda: pcmm.cussen(A, ctB, l, w, k=k, ws=ws), m * l)
            except pcmm.PcmmError as e:
                assert e.status == 2
                continue
            passes += 1
            assert mismatches(got, want) == 0, (k, nb)
    assert passes >= 4


def test_split_gather_over_several_passes(dev):
    # 16 rows x 8 columns give only 32 gather warps, so every output's strips
    # are split over several warps (partial sums added by the combine
    # kernel); smaller workspaces add passes, so the combine also adds onto
    # the previous passes' sums.  Workspaces too small for the partial sums
    # fall back to an unsplit gather.
    m, n, l, w = 16, 200, 8, 4
    pr, A, ctB = _problem(dev, 820, m, n, l, w)
    want = _want(pr)
    full = pcmm.cussen_workspace_bytes(m, n, l, w, 1)
    plan = pcmm.lib().pcmm_cussen_plan_bytes(m, n, w, 1)
    for nb in (full, plan + (full - plan) // 3, plan + (full - plan) // 7, plan + (full - plan) // 40):
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        got = run_affine(lambda: pcmm.cussen(A, ctB, l, w, k=1, ws=ws), m * l)
        assert pcmm.workspace_status(ws) == 0
        assert mismatches(got, want) == 0, nb


def test_workspace_too_small_and_bad_arguments(dev):
    m, n, l, w = 8, 8, 8, 4
    pr, A, ctB = _problem(dev, 900, m, n, l, w)
    ws = torch.empty(1024, dtype=torch.uint8, device=dev)
    with pytest.raises(pcmm.PcmmError) as ei:
        pcmm.cussen(A, ctB, l, w, k=1, ws=ws)
    assert ei.value.status == 2
    ws = pcmm.workspace(m, n, l, w, 1, device=dev)
    with pytest.raises(pcmm.PcmmError) as ei:
        pcmm.cussen(A, ctB, l, w, k=5, ws=ws)      # w * k = 20 > 16
    assert ei.value.status == 1
    with pytest.raises(pcmm.PcmmError):
        pcmm.schoolbook(A, ctB, l, 9)


def test_out_of_range_entries_raise_status(dev):
    m, n, l, w = 8, 6, 4, 3
    pr, A, ctB = _problem(dev, 901, m, n, l, w)
    A2 = A.clone()
    A2[3, 2] = 200                           # >= 2^w
    ws = pcmm.workspace(m, n, l, w, 1, device=dev)
    pcmm.cussen(A2, ctB, l, w, k=1, ws=ws)
    assert pcmm.workspace_status(ws) & 1
    pcmm.cussen(A, ctB, l, w, k=1, ws=ws)
    assert pcmm.workspace_status(ws) == 0


@pytest.mark.parametrize("w", [1, 2, 4, 8])
def test_full_size_sampled(dev, w):
    # The benchmark's workload: 1024 x 1024 times Enc(1024 x 256), autotuned k.
    m, n, l = 1024, 1024, 256
    pr, A, ctB = _problem(dev, inputs.SEED_BASE + 2, m, n, l, w)
    k = pcmm.choose_k(m, n, l, w)
    ws = pcmm.workspace(m, n, l, w, k, device=dev)
    jac = pcmm.cussen(A, ctB, l, w, k=k, ws=ws)
    aff = pcmm.normalize(jac, m * l)
    torch.cuda.synchronize()
    assert pcmm.workspace_status(ws) == 0
    got = pcmm.planar_to_ct(pcmm.to_host_words(aff), m * l)
    rng = np.random.default_rng(w)
    pairs = np.stack([rng.integers(0, m, 96), rng.integers(0, l, 96)], axis=1)
    pairs = np.concatenate([pairs, [[0, 0], [m - 1, l - 1], [m - 1, 0], [0, l - 1]]])
    want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"], pairs=pairs)
    idx = pairs[:, 0] * l + pairs[:, 1]
    assert mismatches(got[idx], want) == 0
    # Every output is a point on the curve (or infinity).
    sample = got[rng.integers(0, m * l, 64)]
    for ct in sample:
        assert oracle.on_curve(ct[0]) and oracle.on_curve(ct[1])


@pytest.mark.parametrize("n,w", [(128, 3), (512, 5), (2048, 7), (2048, 1)])
def test_sweep_config_sampled(dev, n, w):
    # The square sweep workload (A n x n, Enc(B) n x n), as bench.py's sweep
    # mode runs it: cost-model k, sampled outputs against the closed form.
    seed = inputs.SEED_BASE + 3
    pr = inputs.pcmm_problem(seed, n, n, n, 1)
    Ah = inputs.plaintext_matrix(seed, n, n, w)
    ctB = encrypt_gpu(dev, pr)
    A = torch.from_numpy(Ah).to(dev)
    k = pcmm.choose_k(n, n, n, w)
    ws = pcmm.workspace(n, n, n, w, k, device=dev)
    aff = pcmm.normalize(pcmm.cussen(A, ctB, n, w, k=k, ws=ws), n * n)
    torch.cuda.synchronize()
    assert pcmm.workspace_status(ws) == 0
    got = pcmm.planar_to_ct(pcmm.to_host_words(aff), n * n)
    rng = np.random.default_rng(n + w)
    pairs = np.stack([rng.integers(0, n, 48), rng.integers(0, n, 48)], axis=1)
    pairs = np.concatenate([pairs, [[0, 0], [n - 1, n - 1]]])
    want = oracle.closed_form(Ah, pr["r"], pr["sk"], pr["B"], pairs=pairs)
    assert mismatches(got[pairs[:, 0] * n + pairs[:, 1]], want) == 0


def test_base_mul_keygen_matches_oracle(dev):
    s = inputs.streams(123)
    sk = inputs.uniform_scalars(s["sk"], (300,))
    sk[0] = oracle.int_to_words(1)
    sk[1] = oracle.int_to_words(Q - 1)
    sk[2] = oracle.int_to_words(Q)            # = 0 mod q -> infinity
    d = pcmm.to_device_words(pcmm.scalars_to_planar(sk), dev)
    pts = pcmm.base_mul(d, 300)
    torch.cuda.synchronize()
    got = pcmm.planar_to_points(pcmm.to_host_words(pts).reshape(4, 300, 4))
    want = oracle.base_mul(sk)
    assert (got == want).all()
    assert (pcmm.public_key(sk[5], device=dev) == oracle.keygen(sk[5])).all()


def test_resident_plan_serves_several_inputs(dev):
    # Plan once (it depends on A only), execute for two Enc(B) of different widths.
    m, n, w, k = 50, 33, 4, 2
    plan = None
    for l, seed in ((7, 1001), (40, 1002)):
        pr = inputs.pcmm_problem(seed, m, n, l, w)
        if plan is None:
            A_host = pr["A"]
            plan = pcmm.Plan(torch.from_numpy(A_host).to(dev), w, k)
        pr["A"] = A_host
        ctB = encrypt_gpu(dev, pr)
        got = run_affine(lambda: plan.execute(ctB, l), m * l)
        assert mismatches(got, _want(pr)) == 0
        # Smaller scratch: more passes, same result.
        ws = torch.empty(plan.exec_bytes(l) // 3 + 256, dtype=torch.uint8, device=dev)
        try:
            got2 = run_affine(lambda: plan.execute(ctB, l, ws=ws), m * l)
            assert mismatches(got2, _want(pr)) == 0
        except pcmm.PcmmError as e:
            assert e.status == 2


def test_copy_columns_packs_and_splits(dev):
    m, n, w = 20, 12, 3
    parts = []
    for l, seed in ((3, 2001), (5, 2002), (1, 2003)):
        pr = inputs.pcmm_problem(seed, m, n, l, w)
        parts.append((pr, encrypt_gpu(dev, pr), l))
    L = sum(p[2] for p in parts)
    batch = torch.empty(32 * n * L, dtype=torch.int32, device=dev)
    off = 0
    for pr, ct, l in parts:
        pcmm.copy_columns(batch, L, off, ct, l, 0, l, 8 * n)
        off += l
    # The packed batch holds each part's ciphertexts in its column range.
    torch.cuda.synchronize()
    packed = pcmm.planar_to_ct(pcmm.to_host_words(batch), n * L).reshape(n, L, 2, 16)
    off = 0
    for pr, ct, l in parts:
        one = pcmm.planar_to_ct(pcmm.to_host_words(ct), n * l).reshape(n, l, 2, 16)
        assert (packed[:, off:off + l] == one).all()
        # Split back.
        back = torch.empty_like(ct)
        pcmm.copy_columns(back, l, 0, batch, L, off, l, 8 * n)
        torch.cuda.synchronize()
        assert torch.equal(back, ct)
        off += l
