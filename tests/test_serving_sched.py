"""Scheduling logic of the continuous-batching server, exercised on the CPU
with a fake backend (no GPU): column batching per model, FIFO order,
admission by memory budget, rejection of malformed or oversized requests,
cancellation, the in-flight limit, and results equal alone and in the mix."""
import numpy as np
import pytest

from paper_2504_14497_gb300.serving import Request, Server


class FakeBackend:
    """Completes a batch after `delay` polls; the result of a request is the
    plain integer product A X of its (plaintext) input, so that packing and
    splitting of columns is checked end to end."""

    def __init__(self, delay=2):
        self.delay = delay
        self.launched = []

    def load_model(self, A, w, k):
        return np.asarray(A, dtype=np.int64), int(A.size)

    def batch_bytes(self, info, cols):
        return 1000 * cols

    def launch(self, batch):
        A = batch.model.handle
        packed = np.concatenate([r.ct for r in batch.reqs], axis=1)   # n x L
        res = A @ packed
        off = 0
        for r in batch.reqs:
            r.out = res[:, off:off + r.l]
            off += r.l
        self.launched.append([r.rid for r in batch.reqs])
        return [self.delay]

    def done(self, handle):
        handle[0] -= 1
        return handle[0] < 0

    def synchronize(self):
        pass


def _models(rng):
    return {"big": (rng.integers(0, 16, (6, 5)), 4, 1), "small": (rng.integers(0, 16, (3, 4)), 4, 1)}


def _req(rid, model, n, l, t, rng):
    return Request(rid, model, rng.integers(0, 256, (n, l)), l, arrival=t)


def test_batches_pack_same_model_in_fifo_order():
    rng = np.random.default_rng(0)
    be = FakeBackend()
    srv = Server(be, _models(rng), hbm_budget=1e9, max_inflight=1, max_batch_cols=10)
    reqs = [_req(0, "big", 5, 3, 0, rng), _req(1, "small", 4, 2, 0, rng), _req(2, "big", 5, 4, 0, rng),
            _req(3, "big", 5, 5, 0, rng), _req(4, "small", 4, 1, 0, rng)]
    for r in reqs:
        srv.submit(r)
    while not srv.idle():
        srv.step()
    # First batch: the head's model, every waiting request of it that fits 10 columns.
    assert be.launched[0] == [0, 2]
    assert be.launched[1] == [1, 4]
    assert be.launched[2] == [3]
    for r in reqs:
        A = srv.models[r.model].handle
        assert (r.out == A @ r.ct).all()


def test_inflight_limit_and_memory_admission():
    rng = np.random.default_rng(1)
    be = FakeBackend(delay=3)
    models = _models(rng)
    resident = sum(int(np.asarray(A).size) for A, _, _ in models.values())
    # Room for 6 columns of batches next to the resident plans.
    srv = Server(be, models, hbm_budget=resident + 6000, max_inflight=4, max_batch_cols=8)
    reqs = [_req(i, "big" if i % 2 == 0 else "small", 5 if i % 2 == 0 else 4, 3, 0, rng) for i in range(6)]
    for r in reqs:
        srv.submit(r)
    peak_inflight = peak_used = 0
    while not srv.idle():
        srv.step()
        peak_inflight = max(peak_inflight, len(srv.inflight))
        peak_used = max(peak_used, srv.used)
    assert peak_used <= srv.budget
    assert peak_inflight <= 4
    assert len(srv.completed) == 6 and not srv.rejected
    assert srv.used == srv.resident          # all batch memory returned


def test_rejections_and_cancellation():
    rng = np.random.default_rng(2)
    be = FakeBackend()
    models = _models(rng)
    resident = sum(int(np.asarray(A).size) for A, _, _ in models.values())
    srv = Server(be, models, hbm_budget=resident + 5000, max_inflight=1, max_batch_cols=8)
    bad_model = _req(0, "nope", 5, 1, 0, rng)
    bad_l = _req(1, "big", 5, 9, 0, rng)
    too_big = _req(2, "big", 5, 6, 0, rng)        # 6000 bytes alone > 5000 free
    assert not srv.submit(bad_model) and "unknown model" in bad_model.error
    assert not srv.submit(bad_l) and "outside" in bad_l.error
    assert not srv.submit(too_big) and "budget" in too_big.error
    a, b = _req(3, "big", 5, 2, 0, rng), _req(4, "small", 4, 2, 0, rng)
    srv.submit(a)
    srv.submit(b)
    srv.step()                                    # a starts (one slot)
    assert not srv.cancel(a)                      # already running
    assert srv.cancel(b) and b.error == "cancelled"
    while not srv.idle():
        srv.step()
    assert [r.rid for r in srv.completed] == [3]
    assert len(srv.rejected) == 4


def test_replay_with_arrival_times_and_stats():
    rng = np.random.default_rng(3)
    be = FakeBackend(delay=1)
    ticks = iter(range(10**6))
    clock = lambda: next(ticks) * 1e-3            # 1 ms per clock read
    srv = Server(be, _models(rng), hbm_budget=1e9, max_inflight=2, max_batch_cols=16, clock=clock)
    reqs = [_req(i, "big" if i % 3 else "small", 5 if i % 3 else 4, 1 + i % 4, 0.005 * i, rng)
            for i in range(20)]
    done = srv.run(reqs)
    assert len(done) == 20
    st = srv.stats()
    assert st["completed"] == 20 and st["p99_ms"] >= st["p50_ms"] > 0
    for r in reqs:
        assert r.finish >= r.start >= r.arrival
        assert (r.out == srv.models[r.model].handle @ r.ct).all()
