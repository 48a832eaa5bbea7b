"""The persistent batched launch: uneven instances (shapes, bit-widths,
strip widths, several passes with alternating table buffers) give the same
outputs as one pcmm_cussen call per instance and as the CPU oracle, on
repeated runs and when replayed from a captured CUDA graph."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import device, encrypt_gpu, mismatches

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SPECS = [  # m, n, l, w, k
    (37, 70, 20, 3, 1),     # 70 strips: several passes when max_strips is small
    (64, 40, 45, 8, 1),
    (9, 33, 5, 1, 6),
    (50, 21, 33, 4, 2),
    (1, 17, 3, 2, 0),
    (70, 12, 1, 6, 2),
    (16, 16, 16, 4, 3),
    (33, 25, 100, 5, 1),    # 8 table warps per strip: blocks of four share inversions
]


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def batch_case(dev):
    items, probs = [], []
    for i, (m, n, l, w, k) in enumerate(SPECS):
        pr = inputs.pcmm_problem(3100 + i, m, n, l, w)
        ctB = encrypt_gpu(dev, pr)
        A = torch.from_numpy(pr["A"]).to(dev)
        items.append((A, ctB, l, w, k))
        probs.append(pr)
    return items, probs


def _affine(jac, count):
    out = pcmm.normalize(jac, count)
    torch.cuda.synchronize()
    return pcmm.planar_to_ct(pcmm.to_host_words(out), count)


@pytest.mark.parametrize("max_strips", [0, 16, 7])
def test_batched_equals_single_and_oracle(dev, batch_case, max_strips):
    # 16 and 7 strips per pass: five and ten passes for the 70-strip instance,
    # so table buffers are reused and gathers wait across passes.
    items, probs = batch_case
    b = pcmm.Batch(items, max_strips=max_strips)
    outs = b.run()
    torch.cuda.synchronize()
    assert pcmm.workspace_status(b.ws) == 0
    for (A, ctB, l, w, k), pr, out in zip(items, probs, outs):
        m = A.shape[0]
        single = _affine(pcmm.cussen(A, ctB, l, w, k=k), m * l)
        got = _affine(out, m * l)
        assert np.array_equal(got, single)
        want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"]).reshape(-1, 2, 16)
        assert mismatches(got, want) == 0
    # A second run (queue and counters reset) gives the same bytes.
    first = [o.clone() for o in outs]
    b.run()
    torch.cuda.synchronize()
    assert pcmm.workspace_status(b.ws) == 0
    for o, f, (A, _, l, _, _) in zip(b.outs, first, items):
        assert np.array_equal(_affine(o, A.shape[0] * l), _affine(f, A.shape[0] * l))


def test_batched_run_replays_from_a_cuda_graph(dev, batch_case):
    items, _ = batch_case
    b = pcmm.Batch(items)
    b.run()
    torch.cuda.synchronize()
    ref = [_affine(o, A.shape[0] * l) for o, (A, _, l, _, _) in zip(b.outs, items)]
    for o in b.outs:
        o.fill_(0)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.run()
    torch.cuda.synchronize()
    for rep in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert pcmm.workspace_status(b.ws) == 0
        for o, r, (A, _, l, _, _) in zip(b.outs, ref, items):
            assert np.array_equal(_affine(o, A.shape[0] * l), r), rep


def test_autotuner_picks_a_valid_width_and_caches(dev, tmp_path):
    from paper_2504_14497_gb300 import autotune

    path = str(tmp_path / "tune.json")
    k = autotune.tune(96, 64, 40, 4, device=dev, path=path)
    assert k in autotune.candidates(96, 64, 40, 4)
    cache = autotune.load_cache(path)
    assert cache["96,64,40,4"]["k"] == k and len(cache["96,64,40,4"]["ms"]) >= 2
    assert autotune.tune(96, 64, 40, 4, device=dev, path=path) == k   # served from the cache


def test_pass_sizes_per_instance_and_schedule_tuning(dev, batch_case, tmp_path):
    # Explicit strips per pass for every instance (several passes each for
    # the longer ones) give the same outputs as the library's passes; the
    # schedule tuner returns a valid pass size and caches it.
    from paper_2504_14497_gb300 import autotune

    items, probs = batch_case
    ref = pcmm.Batch(items)
    ref_outs = ref.run()
    torch.cuda.synchronize()
    for strips in (1, 3, 5):
        b = pcmm.Batch([it + (strips,) for it in items])
        outs = b.run()
        torch.cuda.synchronize()
        assert pcmm.workspace_status(b.ws) == 0
        for o, r, (A, _, l, _, _) in zip(outs, ref_outs, items):
            assert np.array_equal(_affine(o, A.shape[0] * l), _affine(r, A.shape[0] * l)), strips
    path = str(tmp_path / "tune.json")
    sched = autotune.tune_schedule(96, 200, 40, 4, device=dev, path=path)
    k = sched["k"]
    assert k in autotune.candidates(96, 200, 40, 4)
    assert sched["strips"] == 0 or sched["strips"] in autotune.strip_candidates(96, 200, 40, 4, k)
    assert autotune.load_cache(path)["96,200,40,4"]["strips"] == sched["strips"]
    assert autotune.tune_schedule(96, 200, 40, 4, device=dev, path=path) == sched
    # A workspace sized for a pass of S strips runs S strips per pass: the
    # product is unchanged.
    pr = inputs.pcmm_problem(3300, 37, 70, 20, 3)
    A = torch.from_numpy(pr["A"]).to(dev)
    ctB = encrypt_gpu(dev, pr)
    want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"]).reshape(-1, 2, 16)
    for S in (1, 9, 70):
        ws = torch.empty(pcmm.cussen_workspace_bytes_for(37, 70, 20, 3, 1, S), dtype=torch.uint8, device=dev)
        assert mismatches(_affine(pcmm.cussen(A, ctB, 20, 3, k=1, ws=ws), 37 * 20), want) == 0, S


def test_bounded_wait_gives_up_and_reports(dev):
    import time

    ctr = torch.zeros(1, dtype=torch.int32, device=dev)       # nothing ever sets it
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.full((8,), -1, dtype=torch.int32, device=dev)
    t0 = time.perf_counter()
    pcmm.test_wait(ctr, 1, status, out, 8)
    torch.cuda.synchronize()
    took = time.perf_counter() - t0
    assert int(status.item()) & 4                      # timeout bit raised
    assert (out == 0).all()                            # every warp gave up
    assert took < 30
    # The context is still usable, and a satisfied wait returns at once.
    ctr.fill_(3)
    status.zero_()
    pcmm.test_wait(ctr, 2, status, out, 8)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and (out == 1).all()


def test_batched_workload_config_sampled(dev):
    # The batched workload's 64 shapes (m, n, l uniform in [32, 768], w in
    # 1..8, the same shape seed as the benchmark) in one persistent launch
    # with cost-model strip widths; sampled outputs of every instance against
    # the closed form.
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
    rng = np.random.default_rng(64)
    for (A, _, l, w, _), pr, out in zip(items, probs, outs):
        m = A.shape[0]
        got = _affine(out, m * l)
        pairs = np.stack([rng.integers(0, m, 3), rng.integers(0, l, 3)], axis=1)
        pairs = np.concatenate([pairs, [[0, 0], [m - 1, l - 1]]])
        want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"], pairs=pairs)
        assert mismatches(got[pairs[:, 0] * l + pairs[:, 1]], want) == 0, (m, A.shape[1], l, w)
