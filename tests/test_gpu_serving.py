"""The continuous-batching server on the GPU: each request's result is
bit-identical whether it runs alone or packed with others in a mix of
models, widths and overlapping arrivals, and every output of every request
matches the CPU oracle (small models, and the serving workload's MLP
shapes 256 x 784, 128 x 256 and 10 x 128 with 4-bit weights)."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from paper_2504_14497_gb300.serving import GpuBackend, Request, Server

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_results_identical_alone_and_in_the_mix():
    be = GpuBackend("cuda:0", max_inflight=4)
    dev = be.device
    rng = np.random.default_rng(11)
    shapes = {"a": (40, 70), "b": (24, 33), "c": (5, 20)}
    models = {nm: (rng.integers(0, 16, size=s, dtype=np.uint8), 4, 0) for nm, s in shapes.items()}
    srv = Server(be, models, hbm_budget=4e9, max_inflight=4, max_batch_cols=24)
    s = inputs.streams(77)
    sk = inputs.uniform_scalars(s["sk"], (1,))[0]
    tab = pcmm.keytable(pcmm.public_key(sk, device=dev), device=dev)
    reqs, plain = [], []
    for i in range(36):
        nm = ["a", "b", "c"][i % 3]
        n = shapes[nm][1]
        l = int(rng.integers(1, 9))
        msg = s["B"].integers(0, 256, size=(n, l), dtype=np.uint8)
        r = inputs.uniform_scalars(s["r"], (n, l))
        ct = pcmm.encrypt_table(tab, torch.from_numpy(msg.reshape(-1)).to(dev),
                          pcmm.to_device_words(pcmm.scalars_to_planar(r), dev))
        reqs.append(Request(i, nm, ct, l, arrival=0.0005 * (i // 6)))
        plain.append((msg, r))
    torch.cuda.synchronize()
    srv.run(reqs)
    assert len(srv.completed) == 36 and not srv.rejected
    assert srv.stats()["batches"] < 36            # requests were packed together
    for req, (msg, r) in zip(reqs, plain):
        info = srv.models[req.model]
        A_dev, plan = info.handle
        alone = pcmm.normalize(plan.execute(req.ct, req.l), info.m * req.l)
        torch.cuda.synchronize()
        assert torch.equal(alone, req.out), req.rid
    # Every request against the oracle's closed form.
    for req, (msg, r) in zip(reqs, plain):
        A = models[req.model][0]
        want = oracle.closed_form(A, r, sk, msg).reshape(-1, 2, 16)
        got = pcmm.planar_to_ct(pcmm.to_host_words(req.out), A.shape[0] * req.l)
        assert np.array_equal(got, want)


def test_mlp_shapes_every_output():
    be = GpuBackend("cuda:0", max_inflight=8)
    dev = be.device
    rng = np.random.default_rng(12)
    shapes = {"mlp_784": (256, 784), "mlp_256": (128, 256), "mlp_out": (10, 128)}
    models = {nm: (rng.integers(0, 16, size=sh, dtype=np.uint8), 4, 0) for nm, sh in shapes.items()}
    srv = Server(be, models, hbm_budget=40e9, max_inflight=8, max_batch_cols=256)
    s = inputs.streams(78)
    sk = inputs.uniform_scalars(s["sk"], (1,))[0]
    H = pcmm.public_key(sk, device=dev)
    reqs, plain = [], []
    for i in range(12):
        nm = list(shapes)[i % 3]
        n = shapes[nm][1]
        l = int(rng.integers(1, 65))
        msg = s["B"].integers(0, 256, size=(n, l), dtype=np.uint8)
        r = inputs.uniform_scalars(s["r"], (n, l))
        ct = pcmm.encrypt(H, torch.from_numpy(msg.reshape(-1)).to(dev),
                          pcmm.to_device_words(pcmm.scalars_to_planar(r), dev))
        reqs.append(Request(i, nm, ct, l, arrival=0.0002 * i))
        plain.append((msg, r))
    torch.cuda.synchronize()
    srv.run(reqs)
    assert len(srv.completed) == 12 and not srv.rejected
    for req, (msg, r) in zip(reqs, plain):
        A = models[req.model][0]
        want = oracle.closed_form(A, r, sk, msg).reshape(-1, 2, 16)
        got = pcmm.planar_to_ct(pcmm.to_host_words(req.out), A.shape[0] * req.l)
        assert np.array_equal(got, want), req.rid
