"""Continuous-batching server for encrypted linear layers (PC-MM requests).

A request asks for ``A_model (x) Enc(X)``: a resident plaintext weight matrix
(unsigned w-bit, m x n) times a client's encrypted input batch of l column
vectors (EC-ElGamal over P-256, the paper's encrypted-inference setting,
Sections 1 and 4.3).  The server

* keeps, per model, the plaintext matrix and its Cussen plan (the
  compression of every column of A, Algorithm 3 step 3) resident on the
  device: a request only runs the table build and gather;
* batches continuously: whenever a stream slot is free it takes the oldest
  waiting request and every other waiting request for the same model (in
  arrival order, up to ``max_batch_cols`` columns), packs their ciphertext
  columns into one Enc(B) (columns are independent outputs), runs one
  execution, and splits the result back; requests arriving meanwhile wait
  for the next free slot, so new work joins as slots and memory free up;
* runs up to ``max_inflight`` batches concurrently on separate CUDA streams,
  so their work overlaps on the device;
* admits a batch only while the device memory it needs (scratch, packed
  input, outputs) fits next to the resident plans in ``hbm_budget`` bytes.

All compute runs in libpcmm's kernels; this module is scheduling and
bookkeeping.  A backend object isolates the device calls, so the scheduling
logic can be exercised without a GPU.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Optional


@dataclass
class Request:
    rid: int
    model: str
    ct: object                 # affine ciphertext matrix n x l (backend's array type)
    l: int
    arrival: float = 0.0       # server clock, seconds
    out: object = None         # affine ciphertext matrix m x l, set on completion
    start: Optional[float] = None
    finish: Optional[float] = None
    error: Optional[str] = None
    cancelled: bool = False
    batch_id: Optional[int] = None

    @property
    def latency(self) -> Optional[float]:
        return None if self.finish is None else self.finish - self.arrival


@dataclass
class ModelInfo:
    name: str
    m: int
    n: int
    w: int
    k: int
    handle: object = None      # backend's resident plan
    resident_bytes: int = 0


@dataclass
class Batch:
    bid: int
    model: ModelInfo
    reqs: list
    cols: int
    nbytes: int
    slot: int
    handle: object = None      # backend's completion handle


class GpuBackend:
    """Device calls of the server (libpcmm through its Python binding)."""

    def __init__(self, device="cuda:0", max_inflight: int = 8):
        import torch

        from . import build, pcmm

        build.build()
        self.torch = torch
        self.pcmm = pcmm
        self.device = torch.device(device)
        idx = self.device.index or 0
        torch.cuda.set_device(self.device)
        pcmm.init(idx)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(max_inflight)]

    def load_model(self, A_host, w: int, k: int):
        A = self.torch.from_numpy(A_host).to(self.device)
        plan = self.pcmm.Plan(A, w, k)
        self.torch.cuda.synchronize()
        return (A, plan), int(A.numel() + plan.buf.numel())

    def batch_bytes(self, info: ModelInfo, cols: int) -> int:
        ex = int(self.pcmm.lib().pcmm_cussen_exec_bytes(info.m, info.n, cols, info.w, info.k))
        return ex + 128 * info.n * cols + (192 + 128) * info.m * cols

    def launch(self, batch: Batch):
        torch, pcmm = self.torch, self.pcmm
        info = batch.model
        A, plan = info.handle
        s = self.streams[batch.slot]
        L = batch.cols
        with torch.cuda.stream(s):
            ws = torch.empty(plan.exec_bytes(L), dtype=torch.uint8, device=self.device)
            packed = torch.empty(32 * info.n * L, dtype=torch.int32, device=self.device)
            jac = torch.empty(48 * info.m * L, dtype=torch.int32, device=self.device)
            aff = torch.empty(32 * info.m * L, dtype=torch.int32, device=self.device)
            off = 0
            for r in batch.reqs:
                pcmm.copy_columns(packed, L, off, r.ct, r.l, 0, r.l, 8 * info.n, stream=s)
                off += r.l
            plan.execute(packed, L, ws=ws, out=jac, stream=s)
            pcmm.normalize(jac, info.m * L, out=aff, stream=s)
            off = 0
            for r in batch.reqs:
                r.out = torch.empty(32 * info.m * r.l, dtype=torch.int32, device=self.device)
                pcmm.copy_columns(r.out, r.l, 0, aff, L, off, r.l, 8 * info.m, stream=s)
                off += r.l
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, ws, packed, jac, aff)

    def done(self, handle) -> bool:
        return handle[0].query()

    def synchronize(self):
        self.torch.cuda.synchronize()


class Server:
    def __init__(self, backend, models: dict, hbm_budget: float = 40e9, max_inflight: int = 8,
                 max_batch_cols: int = 256, clock=time.perf_counter):
        """models: name -> (A_host uint8 m x n, w, k); k = 0 picks the strip
        width for a full batch with the library's cost model."""
        self.backend = backend
        self.budget = float(hbm_budget)
        self.max_inflight = int(max_inflight)
        self.max_cols = int(max_batch_cols)
        self.clock = clock
        self.models = {}
        self.used = 0
        for name, (A, w, k) in models.items():
            m, n = A.shape
            if not k:
                k = self._choose_k(m, n, self.max_cols, w)
            info = ModelInfo(name, m, n, int(w), int(k))
            info.handle, info.resident_bytes = backend.load_model(A, int(w), int(k))
            self.used += info.resident_bytes
            self.models[name] = info
        if self.used > self.budget:
            raise MemoryError("resident plans exceed the HBM budget")
        self.resident = self.used
        self.waiting = collections.deque()
        self.inflight = []
        self.free_slots = list(range(self.max_inflight))
        self.completed = []
        self.rejected = []
        self._bid = 0
        self.t0 = self.clock()

    def _choose_k(self, m, n, l, w):
        try:
            from . import pcmm
            return pcmm.choose_k(m, n, l, w)
        except Exception:  # backends without the library (scheduling tests)
            return 1

    def now(self) -> float:
        return self.clock() - self.t0

    # ------------------------------------------------------------ admission
    def submit(self, req: Request) -> bool:
        info = self.models.get(req.model)
        if info is None:
            req.error = f"unknown model {req.model!r}"
        elif not 1 <= req.l <= self.max_cols:
            req.error = f"l = {req.l} outside [1, {self.max_cols}]"
        elif self.backend.batch_bytes(info, req.l) + self.resident > self.budget:
            req.error = "request alone exceeds the HBM budget"
        if req.error:
            req.finish = self.now()
            self.rejected.append(req)
            return False
        self.waiting.append(req)
        return True

    def cancel(self, req: Request) -> bool:
        """Cancels a request that has not started; returns False otherwise."""
        if req.start is None and not req.cancelled and req in self.waiting:
            req.cancelled = True
            self.waiting.remove(req)
            req.error = "cancelled"
            req.finish = self.now()
            self.rejected.append(req)
            return True
        return False

    # ------------------------------------------------------------- schedule
    def _form_batch(self):
        head = self.waiting[0]
        info = self.models[head.model]
        take, cols = [], 0
        for r in self.waiting:
            if r.model == head.model and cols + r.l <= self.max_cols:
                take.append(r)
                cols += r.l
        return info, take, cols

    def step(self) -> int:
        """Retires finished batches and launches new ones; returns the number
        of batches launched."""
        now = self.now()
        still = []
        for b in self.inflight:
            if self.backend.done(b.handle):
                for r in b.reqs:
                    r.finish = now
                    self.completed.append(r)
                self.used -= b.nbytes
                self.free_slots.append(b.slot)
            else:
                still.append(b)
        self.inflight = still
        launched = 0
        while self.free_slots and self.waiting:
            info, take, cols = self._form_batch()
            need = self.backend.batch_bytes(info, cols)
            if self.used + need > self.budget:
                # Shrink to what fits; if even the head does not fit, wait for memory.
                while len(take) > 1 and self.used + need > self.budget:
                    cols -= take.pop().l
                    need = self.backend.batch_bytes(info, cols)
                if self.used + need > self.budget:
                    break
            slot = self.free_slots.pop()
            b = Batch(self._bid, info, take, cols, need, slot)
            self._bid += 1
            for r in take:
                self.waiting.remove(r)
                r.start = now
                r.batch_id = b.bid
            b.handle = self.backend.launch(b)
            self.used += need
            self.inflight.append(b)
            launched += 1
        return launched

    def idle(self) -> bool:
        return not self.waiting and not self.inflight

    def run(self, requests, poll_sleep: float = 0.0, timeout: float = 600.0):
        """Replays requests at their arrival times (server clock) until all
        are finished or rejected."""
        pending = sorted(requests, key=lambda r: r.arrival)
        i = 0
        self.t0 = self.clock()
        while i < len(pending) or not self.idle():
            now = self.now()
            if now > timeout:
                raise TimeoutError("serving run exceeded its timeout")
            while i < len(pending) and pending[i].arrival <= now:
                self.submit(pending[i])
                i += 1
            self.step()
            if poll_sleep:
                time.sleep(poll_sleep)
        self.backend.synchronize()
        return self.completed

    # -------------------------------------------------------------- metrics
    def stats(self) -> dict:
        lat = sorted(r.latency for r in self.completed if r.latency is not None)
        if not lat:
            return {"completed": 0, "rejected": len(self.rejected)}

        def pct(q):
            return lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]

        first = min(r.arrival for r in self.completed)
        last = max(r.finish for r in self.completed)
        return {"completed": len(lat), "rejected": len(self.rejected),
                "p50_ms": 1e3 * pct(0.50), "p99_ms": 1e3 * pct(0.99),
                "mean_ms": 1e3 * sum(lat) / len(lat),
                "req_per_s": len(lat) / max(last - first, 1e-9),
                "batches": self._bid}
