#!/usr/bin/env python
"""Throughput benchmark of encrypted PC-MM (Cussen's method) on GB300.

Workload (one step): the single large PC-MM, A 1024 x 1024 with unsigned
w-bit entries for each w in {1, 2, 4, 8}, times Enc(B) 1024 x 256 (8-bit
messages, EC-ElGamal over P-256), Cussen with the cost model's strip width,
followed by affine normalisation of the 1024 x 256 output ciphertexts.
Inputs are seeded and synthetic.  The metric is point additions (of two
finite points, including the doublings of the compressed-value
multiplications) performed per second; the dominant kernel's rate is also
reported against the integer multiply-add (IMAD) roofline.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs the same workload on its own GPU
(replicas, no collective on the data path) and rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "encrypted PC-MM ciphertext point-adds/s and % int/HBM roofline (bit-exact) vs plain"
UNIT = "point-adds/s"
SEED = 2504144970 + 2         # the large single PC-MM workload


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--widths", default="1,2,4,8")
    ap.add_argument("--shape", default="1024,1024,256", help="m,n,l")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-schoolbook", action="store_true")
    ap.add_argument("--workload", choices=["large", "serving", "batched", "sweep", "vector", "decrypt", "sparse",
                                           "strassen"],
                    default="large",
                    help="large: the single large PC-MM (the headline line); serving: Poisson "
                         "request sweep of encrypted linear layers; batched: 64 uneven instances; "
                         "sweep: square PC-MM over n and w, Cussen beside schoolbook; vector: "
                         "plaintext vector times ciphertext scalars; decrypt: baby-step "
                         "giant-step decryption of the large w = 8 product's output; sparse: the "
                         "large product with mostly-zero A; strassen: schoolbook, Strassen and Cussen "
                         "on square products (the paper's comparison)")
    ap.add_argument("--sweep-n", default="128,256,512,1024,2048")
    ap.add_argument("--strassen-n", default="128,256,512,1024")
    ap.add_argument("--strassen-widths", default="4,8,12,16")
    ap.add_argument("--sweep-widths", default="1,2,3,4,5,6,7,8,12,16")
    ap.add_argument("--vector-n", default="8,16,32,64,128,256,512")
    ap.add_argument("--vector-widths", default="4,8,12,16")
    ap.add_argument("--vector-scalars", type=int, default=65536)
    ap.add_argument("--sparse-densities", default="1,0.5,0.2,0.1,0.05,0.02,0.01")
    ap.add_argument("--sparse-widths", default="8,4")
    ap.add_argument("--rates", default="10,20,50,100,200,500,1000,2000")
    ap.add_argument("--seconds", type=float, default=2.0, help="arrival window per rate (serving)")
    ap.add_argument("--serving-inflight", type=int, default=8, help="batches in flight (serving)")
    ap.add_argument("--serving-cols", type=int, default=256, help="columns per batch at most (serving)")
    return ap.parse_args()


# ------------------------------------------------------------ distributed

class Dist:
    def __init__(self, gpus):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo", rank=self.rank, world_size=self.world)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def replica_rate(world: int, units_per_rank: float, steps: int, max_ms: float) -> float:
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units per step for `steps` steps, timed by the slowest
    rank (max_ms over ranks)."""
    return world * units_per_rank * steps / (max_ms / 1e3)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.sw_power_cap,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["sw_power_cap", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- workload

def recorded_profile(kernel: str):
    """The committed ncu record of `kernel` in profiles/ (a JSON block with
    per-launch DRAM traffic scaled to the headline launch and the kernel's
    instruction mix per unit of work), or None when the kernel's source has
    changed since it was taken."""
    import glob
    import hashlib
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read()
        if "```json" not in text:
            continue
        rec = json.loads(text.split("```json", 1)[1].split("```", 1)[0])
        if rec.get("kernel") != kernel:
            continue
        h = hashlib.sha256()
        for f in rec["source_files"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() == rec["source_sha256"]:
            return rec
    return None


def measure_peaks(dev, repeats: int = 5) -> dict:
    """Measured integer-pipe peaks of this GPU (thread-level instructions per
    second): independent mad.lo / mad.hi / mad.wide / add.cc-addc / add
    streams over whole waves of all SMs, best of `repeats` CUDA-event timings
    after a warm-up launch.  mul.wide.u32 and mad.wide.u32 each form one
    32 x 32 -> 64-bit limb product; the faster of the two streams is the
    product peak (a mad.wide chain whose multiplicand and accumulator both
    come from 64-bit results measured at about a third of the mul.wide
    rate)."""
    import torch

    from paper_2504_14497_gb300 import pcmm
    props = torch.cuda.get_device_properties(dev)
    blocks = props.multi_processor_count * 4
    sink = torch.zeros(1024, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    for op, iters in (("mad_lo", 200000), ("mad_hi", 100000), ("mad_wide", 100000), ("mul_wide", 200000),
                      ("add_carry", 200000), ("add", 200000)):
        pcmm.peak_run(op, blocks, 2000, sink)
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ops = pcmm.peak_run(op, blocks, iters, sink)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[op] = ops / (best / 1e3)
    out["product"] = max(out["mad_wide"], out["mul_wide"])
    out["sms"] = props.multi_processor_count
    return out


def _host_plaintext(A):
    """Host tensor of a plaintext matrix: uint8, or int16 holding the bits of
    a uint16 matrix (entries of more than 8 bits)."""
    import torch
    return torch.from_numpy(A.view(np.int16) if A.dtype == np.uint16 else A)


def make_problem(m, n, l, widths):
    from paper_2504_14497_gb300 import inputs
    pr = {w: inputs.pcmm_problem(SEED, m, n, l, w) for w in widths}
    return pr


_CPU_CT = {}


def cpu_sample(problem, w, m_s, l_s, k):
    """The CPU oracle on a bounded sample of the workload: the first m_s rows
    of A and the first l_s columns of Enc(B) (encrypted by the oracle, once,
    outside the timing).  Returns (point additions, seconds)."""
    from oracle import oracle
    A = problem["A"][:m_s]
    key = (id(problem), l_s)
    if key not in _CPU_CT:
        H = oracle.keygen(problem["sk"])
        _CPU_CT[key] = oracle.encrypt(H, problem["B"][:, :l_s], problem["r"][:, :l_s])
    ct = _CPU_CT[key]
    t0 = time.perf_counter()
    _, cnt = oracle.cussen(A, ct, w, k)
    dt = time.perf_counter() - t0
    adds = cnt["ecsm_dbl"] + cnt["ecsm_add"] + cnt["recon_add"] + cnt["accum_add"]
    return adds, dt


def run_reference(args, dist):
    """The CPU oracle as it stands, timed on the host cores."""
    m, n, l = (int(x) for x in args.shape.split(","))
    if dist.rank != 0:
        return None
    from oracle import oracle
    from paper_2504_14497_gb300 import inputs
    w, m_s, l_s, k = 4, 64, 16, 2
    problem = inputs.pcmm_problem(SEED, m, n, l, w)
    for _ in range(args.warmup):
        cpu_sample(problem, w, m_s, l_s, k)
    adds_tot, sec_tot = 0, 0.0
    for _ in range(args.steps):
        a, s = cpu_sample(problem, w, m_s, l_s, k)
        adds_tot += a
        sec_tot += s
    value = adds_tot / sec_tot
    sample = f"w=4 k=2 Cussen, rows 0..{m_s - 1} x Enc(B) columns 0..{l_s - 1} of the {m}x{n}x{l} workload"
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded)",
        "config": {"workload": f"single large PC-MM {m}x{n}x{l}, CPU oracle sample", "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_ours(args, dist):
    import torch

    from paper_2504_14497_gb300 import build, counts, pcmm

    build.build()
    dev_index = dist.local if torch.cuda.device_count() > dist.local else 0
    torch.cuda.set_device(dev_index)
    dev = torch.device("cuda", dev_index)
    pcmm.init(dev_index)
    m, n, l = (int(x) for x in args.shape.split(","))
    widths = [int(x) for x in args.widths.split(",")]
    problems = make_problem(m, n, l, widths)
    base = problems[widths[0]]
    H = pcmm.public_key(base["sk"], device=dev)
    tab = pcmm.keytable(H, device=dev)
    msg = torch.from_numpy(base["B"].reshape(-1)).to(dev)
    rr = pcmm.to_device_words(pcmm.scalars_to_planar(base["r"]), dev)
    ctB = pcmm.encrypt_table(tab, msg, rr)
    stream = torch.cuda.current_stream()
    runs = []
    for w in widths:
        k = pcmm.choose_k(m, n, l, w)
        A = _host_plaintext(problems[w]["A"]).to(dev)
        ws = pcmm.workspace(m, n, l, w, k, device=dev)
        jac = torch.empty(48 * m * l, dtype=torch.int32, device=dev)
        aff = torch.empty(32 * m * l, dtype=torch.int32, device=dev)
        c = counts.cussen_counts(problems[w]["A"], w, k, l)
        runs.append(dict(w=w, k=k, A=A, ws=ws, jac=jac, aff=aff, counts=c))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        for r in runs:
            pcmm.cussen(r["A"], ctB, l, r["w"], k=r["k"], ws=r["ws"], out=r["jac"])
            pcmm.normalize(r["jac"], m * l, out=r["aff"])

    # Integer-pipe peaks (outside the timed region), with the clocks seen.
    pclk = ClockSampler(dev_index)
    pclk.start()
    peaks = measure_peaks(dev)
    peak_clk = pclk.stop()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for r in runs:
        if pcmm.workspace_status(r["ws"]) != 0:
            raise RuntimeError("device status word set during warm-up")

    # ---- timed region: K steps, L2 flushed between steps (outside events)
    clocks = ClockSampler(dev_index)
    pcmm.profile_enable(64 * args.steps * len(widths) + 64)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    clk = clocks.stop()
    dist.barrier()
    prof = pcmm.profile_read()
    pcmm.profile_enable(0)
    total_ms = dist.max(total_ms)

    ops_step = sum(counts.point_ops(r["counts"]) for r in runs)
    value = replica_rate(dist.world, ops_step, args.steps, total_ms)
    launches = sum(v[1] for v in prof.values())

    # ---- roofline of the dominant kernel, against the measured peaks:
    # algorithmic limb products per second over the measured mad.wide rate
    # (one product each), and the binding ALU pipe's issue rate (the
    # kernel's ALU instructions per unit of work from its committed ncu
    # record) over the measured add.cc / addc rate.
    props = torch.cuda.get_device_properties(dev)
    prod_peak = peaks["product"]
    alu_peak = peaks["add_carry"]
    prods = {"gather": sum(counts.gather_imad(r["counts"]) for r in runs) // counts.IMAD_PER_PRODUCT,
             "table": sum(counts.table_imad(r["counts"]) for r in runs) // counts.IMAD_PER_PRODUCT}
    units = {"gather": sum(r["counts"]["gather_madd"] for r in runs),
             "table": sum(counts.point_ops(r["counts"]) - r["counts"]["gather_madd"] for r in runs)}
    kernels = {nm: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
               for nm, v in prof.items() if v[1]}
    for nm in ("gather", "table"):
        if nm not in kernels:
            continue
        sec = prof[nm][0] / 1e3
        kernels[nm]["products_per_s"] = prods[nm] * args.steps / sec
        kernels[nm]["frac_product_peak"] = kernels[nm]["products_per_s"] / prod_peak
        # The records' instruction mix was captured at w in {1, 2, 4, 8}.
        rec = recorded_profile(nm) if set(widths) <= {1, 2, 4, 8} else None
        if rec and rec.get("alu_warp_inst_per_unit"):
            alu_rate = units[nm] * args.steps * rec["alu_warp_inst_per_unit"] * 32 / sec
            kernels[nm]["alu_inst_per_s"] = alu_rate
            kernels[nm]["frac_alu_peak"] = alu_rate / alu_peak
    dom = max(("gather", "table"), key=lambda nm: prof[nm][0])
    dom_ms, dom_launches = prof[dom]
    # The recorded traffic is per launch of the 1024 x 1024 x 256 step at w in {1, 2, 4, 8}.
    rec = recorded_profile(dom) if (m, n, l) == (1024, 1024, 256) and sorted(widths) == [1, 2, 4, 8] else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": kernels[dom]["products_per_s"] / 1e12,
                "peak": prod_peak / 1e12, "unit": "T limb-products/s",
                "frac": kernels[dom]["frac_product_peak"],
                "traffic": rec.get("traffic_bytes_per_launch") if rec else None,
                "launches": dom_launches, "avg_launch_ms": dom_ms / max(dom_launches, 1),
                "peak_basis": "measured: faster of the mul.wide.u32 / mad.wide.u32 streams (one "
                              f"32x32->64-bit product each) over {props.multi_processor_count} SMs in this run",
                "alu_frac": kernels[dom].get("frac_alu_peak"),
                "alu_peak": alu_peak / 1e12, "alu_unit": "T thread-inst/s (add.cc/addc, measured)",
                "peaks_measured": {k: (v / 1e12 if k != "sms" else v) for k, v in peaks.items()},
                "peaks_clocks": peak_clk}

    # ---- schoolbook on the same GPU (context: Cussen speed-up, w = 8 and 4)
    schoolbook = None
    if not args.no_schoolbook and dist.rank == 0:
        schoolbook = {}
        for r in runs:
            if r["w"] not in (4, 8):
                continue
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            pcmm.schoolbook(r["A"], ctB, l, r["w"], out=r["jac"])
            ev1.record(stream)
            ev1.synchronize()
            ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev2.record(stream)
            pcmm.cussen(r["A"], ctB, l, r["w"], k=r["k"], ws=r["ws"], out=r["jac"])
            ev3.record(stream)
            ev3.synchronize()
            sb, cu = ev0.elapsed_time(ev1), ev2.elapsed_time(ev3)
            schoolbook[f"w{r['w']}"] = {"schoolbook_ms": sb, "cussen_ms": cu, "speedup": sb / cu}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        hA = [_host_plaintext(problems[r["w"]]["A"]).pin_memory() for r in runs]
        hB = pcmm.to_host_words(ctB).view(np.int32)
        hB = torch.from_numpy(hB.copy()).pin_memory()
        hC = [torch.empty(32 * m * l, dtype=torch.int32).pin_memory() for _ in runs]
        dB = torch.empty_like(ctB)
        dA = [torch.empty_like(r["A"]) for r in runs]

        def e2e_step():
            dB.copy_(hB, non_blocking=True)
            for r, a_h, a_d, c_h in zip(runs, hA, dA, hC):
                a_d.copy_(a_h, non_blocking=True)
                pcmm.cussen(a_d, dB, l, r["w"], k=r["k"], ws=r["ws"], out=r["jac"])
                pcmm.normalize(r["jac"], m * l, out=r["aff"])
                c_h.copy_(r["aff"], non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        dist.barrier()
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            e2e_step()
            ev1.record(stream)
            ev1.synchronize()
            e2e_ms += ev0.elapsed_time(ev1)
        e2e_ms = dist.max(e2e_ms)
        e2e = {"value": replica_rate(dist.world, ops_step, args.steps, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(hB.numel() * 4 + sum(a.numel() for a in hA)),
               "d2h_bytes_per_step": int(sum(c.numel() * 4 for c in hC)),
               "ms_per_step": e2e_ms / args.steps}

    # ---- CPU oracle baseline on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if not args.no_cpu_baseline and dist.world == 1:
        from oracle import oracle
        w_s = 4 if 4 in problems else widths[0]
        m_s, l_s, k_s = 128, 16, pcmm.choose_k(m, n, l, w_s)
        adds, sec = cpu_sample(problems[w_s], w_s, m_s, l_s, k_s)
        cpu = {"value": adds / sec, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
               "sample": f"w={w_s} k={k_s} Cussen on rows 0..{m_s - 1} x Enc(B) columns 0..{l_s - 1}"
                         f" of the {m}x{n}x{l} workload ({adds} point additions, {sec:.1f} s)"}

    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded)",
        "config": {"workload": f"single large PC-MM A {m}x{n} (w in {widths}) x Enc(B) {n}x{l}, "
                               f"EC-ElGamal P-256, Cussen + affine normalisation",
                   "m": m, "n": n, "l": l, "widths": widths,
                   "k": {f"w{r['w']}": r["k"] for r in runs},
                   "l2": "flushed between timed steps (512 MiB write outside the events)",
                   "parallelism": f"replicas x{dist.world}"},
        "point_ops_per_step": ops_step,
        "roofline": roofline, "kernels": kernels, "gpu_launches": launches,
        "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "schoolbook": schoolbook,
    }


def run_batched(args, dist):
    """64 independent PC-MM instances (m, n, l uniform in [32, 768], w uniform
    in {1..8}, 8-bit messages): strip widths and pass sizes from the autotuner
    (the pass size given to each instance of the persistent launch and to its
    plain launch; the library's default passes timed as well), all instances
    in one persistent launch replayed from a CUDA graph, against one plain
    pcmm_cussen launch per instance on the same GPU."""
    import torch

    from paper_2504_14497_gb300 import autotune, build, counts, inputs, pcmm

    build.build()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    pcmm.init(dist.local)
    shapes = inputs.batched_shapes(SEED + 2, count=64)
    st = inputs.streams(SEED + 2)
    sk = inputs.uniform_scalars(st["sk"], (1,))[0]
    tab = pcmm.keytable(pcmm.public_key(sk, device=dev), device=dev)
    cache = {}
    items, ops = [], 0
    t_tune = time.perf_counter()
    strips = []
    for i, (m, n, l, w) in enumerate(shapes):
        sched = autotune.tune_schedule(m, n, l, w, device=dev, cache=cache)
        k = sched["k"]
        strips.append(sched["strips"])
        A_h = st["A"].integers(0, 1 << w, size=(m, n), dtype=np.uint8)
        msg = st["B"].integers(0, 256, size=(n * l,), dtype=np.uint8)
        r = inputs.uniform_scalars(st["r"], (n * l,))
        ctB = pcmm.encrypt_table(tab, torch.from_numpy(msg).to(dev), pcmm.to_device_words(pcmm.scalars_to_planar(r), dev))
        items.append((torch.from_numpy(A_h).to(dev), ctB, l, w, k))
        ops += counts.point_ops(counts.cussen_counts(A_h, w, k, l))
    t_tune = time.perf_counter() - t_tune
    torch.cuda.synchronize()

    def persistent_ms(batch_items):
        """Mean ms of `steps` graph replays of one persistent launch."""
        b = pcmm.Batch(batch_items)
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            for _ in range(max(args.warmup, 1)):
                b.run()
            torch.cuda.synchronize()
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, stream=st):
                b.run()
        torch.cuda.synchronize()
        c = torch.cuda.current_stream()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(c)
        for _ in range(args.steps):
            gr.replay()
        a1.record(c)
        a1.synchronize()
        if pcmm.workspace_status(b.ws) != 0:
            raise RuntimeError("batched run reported a device error")
        return a0.elapsed_time(a1) / args.steps

    # The library's default pass sizes, for context.
    ms_default_schedule = persistent_ms(items)
    items = [it + (S,) for it, S in zip(items, strips)]
    batch = pcmm.Batch(items)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 1)):
            batch.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            batch.run()
    torch.cuda.synchronize()
    if pcmm.workspace_status(batch.ws) != 0:
        raise RuntimeError("batched run reported a device error")
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for _ in range(args.steps):
        g.replay()
    e1.record(cur)
    e1.synchronize()
    ms_batched = e0.elapsed_time(e1) / args.steps
    if pcmm.workspace_status(batch.ws) != 0:
        raise RuntimeError("batched run reported a device error")
    # One plain launch per instance (plan + tables + gather each), same k.
    # The launches run one after another on one stream, so they share one
    # allocation; each gets exactly its default workspace size.
    # Each gets the workspace of its tuned pass size (its default when none was better).
    need = [pcmm.cussen_workspace_bytes_for(A.shape[0], A.shape[1], l, w, k, S) if S
            else pcmm.cussen_workspace_bytes(A.shape[0], A.shape[1], l, w, k) for A, _, l, w, k, S in items]
    shared = torch.empty(max(need), dtype=torch.uint8, device=dev)
    wss = [shared[:nb] for nb in need]
    outs = [torch.empty(48 * it[0].shape[0] * it[2], dtype=torch.int32, device=dev) for it in items]

    def plain():
        for (A, ctB, l, w, k, _), ws, out in zip(items, wss, outs):
            pcmm.cussen(A, ctB, l, w, k=k, ws=ws, out=out)

    plain()
    torch.cuda.synchronize()
    e0.record(cur)
    for _ in range(args.steps):
        plain()
    e1.record(cur)
    e1.synchronize()
    ms_plain = e0.elapsed_time(e1) / args.steps
    same = all(torch.equal(pcmm.normalize(o, A.shape[0] * l), pcmm.normalize(b, A.shape[0] * l))
               for o, b, (A, _, l, _, _, _) in zip(outs, batch.outs, items))
    return {"workload": "batched: 64 PC-MM instances, m,n,l ~ U[32,768], w ~ U{1..8}, 8-bit messages, "
                        "one persistent launch replayed from a CUDA graph",
            "metric": "point-adds/s (batched) vs one launch per instance", "unit": "point-adds/s",
            "value": ops / (ms_batched / 1e3), "ms_per_batch": ms_batched,
            "plain_value": ops / (ms_plain / 1e3), "plain_ms_per_batch": ms_plain,
            "speedup_vs_plain": ms_plain / ms_batched, "point_ops_per_batch": ops,
            "outputs_identical": bool(same), "k": [it[4] for it in items],
            "strips_per_pass": [it[5] for it in items],
            "ms_per_batch_default_schedule": ms_default_schedule,
            "autotune_s": t_tune, "steps": args.steps, "n_gpus": 1}


def run_sweep(args, dist):
    """Square PC-MM sweep: A n x n with uniform w-bit entries times Enc(B)
    n x n (8-bit messages) for every n and w asked for.  Per (n, w): the
    Cussen wall time (cost-model k, best of two calls after a warm-up), its
    point additions per second and IMAD fraction, and the schoolbook wall
    time on the same GPU.  The schoolbook is timed on a slice of rows sized
    to about 4e9 point operations and scaled to n rows: every output row is
    an independent sum of the same cost."""
    import torch

    from paper_2504_14497_gb300 import build, counts, inputs, pcmm

    build.build()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    pcmm.init(dist.local)
    props = torch.cuda.get_device_properties(dev)
    clocks = ClockSampler(dist.local)
    clocks.start()
    seed = 2504144970 + 3
    cur = torch.cuda.current_stream()

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            fn()
            e1.record(cur)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    rows = []
    for n in (int(x) for x in args.sweep_n.split(",")):
        pr = inputs.pcmm_problem(seed, n, n, n, 1)
        tab = pcmm.keytable(pcmm.public_key(pr["sk"], device=dev), device=dev)
        ctB = pcmm.encrypt_table(tab, torch.from_numpy(pr["B"].reshape(-1)).to(dev),
                           pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev))
        out = torch.empty(48 * n * n, dtype=torch.int32, device=dev)
        for w in (int(x) for x in args.sweep_widths.split(",")):
            A_h = inputs.plaintext_matrix(seed, n, n, w)
            A = _host_plaintext(A_h).to(dev)
            k = pcmm.choose_k(n, n, n, w)
            ws = pcmm.workspace(n, n, n, w, k, device=dev)
            ms = timed(lambda: pcmm.cussen(A, ctB, n, w, k=k, ws=ws, out=out))
            if pcmm.workspace_status(ws) != 0:
                raise RuntimeError(f"device status at n={n} w={w}")
            del ws
            c = counts.cussen_counts(A_h, w, k, n)
            ops = counts.point_ops(c)
            imad = counts.gather_imad(c) + counts.table_imad(c)
            ops_row = 2.0 * n * n * (1.5 * w + 1)          # schoolbook point operations per row
            ms_rows = int(min(n, max(8, 4e9 // ops_row)))
            sb = timed(lambda: pcmm.schoolbook(A[:ms_rows], ctB, n, w, out=out), reps=1)
            sb_full = sb * n / ms_rows
            rows.append({"n": n, "w": w, "k": k, "cussen_ms": ms, "point_adds_per_s": ops / (ms / 1e3),
                         "imad": imad, "schoolbook_ms": sb_full,
                         "schoolbook_rows_timed": ms_rows, "speedup_vs_schoolbook": sb_full / ms})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            torch.cuda.empty_cache()
        del ctB, out
        torch.cuda.empty_cache()
    clk = clocks.stop()
    # Measured product peak (mad.wide.u32 rate), two IMAD-equivalents each.
    peak = measure_peaks(dev)["product"] * counts.IMAD_PER_PRODUCT
    for r in rows:
        r["imad_frac"] = r.pop("imad") / (r["cussen_ms"] / 1e3) / peak
    return {"workload": "sweep: square PC-MM A n x n (uniform w-bit) x Enc(B) n x n (8-bit messages), "
                        "Cussen with cost-model k beside schoolbook, one PC-MM per launch",
            "metric": "Cussen PC-MM wall time and point-adds/s per (n, w)", "unit": "ms",
            "peak_imad_per_s": peak, "clocks": clk, "rows": rows, "n_gpus": 1, "data": "synthetic (seeded)"}


def run_strassen(args, dist):
    """The paper's comparison systems on the GPU (Sections 3.1 and 4.2):
    square A n x n (uniform w-bit; uint16 for w > 8) times Enc(B) n x n, schoolbook,
    Strassen PC-MM at every recursion depth from 1 to the one leaving 16 x 16
    leaf blocks (at most 5), and Cussen (cost-model k), each timed as one
    launch sequence with CUDA events (best of two after a warm-up); the
    Strassen and Cussen outputs are checked equal after normalisation.  The
    schoolbook is timed on a row slice scaled to n rows, as in the sweep."""
    import torch

    from paper_2504_14497_gb300 import build, counts, inputs, pcmm

    build.build()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    pcmm.init(dist.local)
    clocks = ClockSampler(dist.local)
    clocks.start()
    seed = 2504144970 + 7
    cur = torch.cuda.current_stream()

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            fn()
            e1.record(cur)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    rows = []
    for n in (int(x) for x in args.strassen_n.split(",")):
        pr = inputs.pcmm_problem(seed, n, n, n, 1)
        ctB = pcmm.encrypt(pcmm.public_key(pr["sk"], device=dev), torch.from_numpy(pr["B"].reshape(-1)).to(dev),
                           pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev))
        out = torch.empty(48 * n * n, dtype=torch.int32, device=dev)
        out2 = torch.empty_like(out)
        for w in (int(x) for x in args.strassen_widths.split(",")):
            A_h = inputs.plaintext_matrix(seed, n, n, w)
            A = _host_plaintext(A_h).to(dev)
            k = pcmm.choose_k(n, n, n, w)
            ws = pcmm.workspace(n, n, n, w, k, device=dev)
            cu = timed(lambda: pcmm.cussen(A, ctB, n, w, k=k, ws=ws, out=out))
            ref = pcmm.normalize(out, n * n)
            del ws
            ops_row = 2.0 * n * n * (1.5 * w + 1)
            ms_rows = int(min(n, max(8, 4e9 // ops_row)))
            sb = timed(lambda: pcmm.schoolbook(A[:ms_rows], ctB, n, w, out=out2), reps=1) * n / ms_rows
            depths = {}
            same = True
            d = 1
            while d <= 5 and (n >> d) >= 16:
                wsb = torch.empty(pcmm.strassen_workspace_bytes(n, n, n, w, d), dtype=torch.uint8, device=dev)
                ms = timed(lambda: pcmm.strassen(A, ctB, n, w, d, ws=wsb, out=out2), reps=1)
                same &= bool(torch.equal(pcmm.normalize(out2, n * n), ref))
                c = counts.strassen_counts(A_h, w, d, n)
                depths[d] = {"ms": ms, "point_adds_per_s": counts.strassen_point_ops(c) / (ms / 1e3)}
                del wsb
                torch.cuda.empty_cache()
                d += 1
            best_d = min(depths, key=lambda x: depths[x]["ms"]) if depths else None
            st_ms = depths[best_d]["ms"] if depths else None
            row = {"n": n, "w": w, "cussen_ms": cu, "cussen_k": k, "schoolbook_ms": sb,
                   "strassen": depths, "strassen_best_depth": best_d, "strassen_ms": st_ms,
                   "speedup_cussen_vs_strassen": st_ms / cu if st_ms else None,
                   "speedup_cussen_vs_schoolbook": sb / cu,
                   "speedup_strassen_vs_schoolbook": sb / st_ms if st_ms else None,
                   "paper_equiv_adds": {"schoolbook": 2 * n ** 3 * 2 * w + 2 * n * n * (n - 1),
                                        "strassen": counts.strassen_equiv(n, w)},
                   "outputs_identical": same}
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
            torch.cuda.empty_cache()
        del ctB, out, out2
        torch.cuda.empty_cache()
    clk = clocks.stop()
    return {"workload": "strassen: square PC-MM A n x n (uniform w-bit) x Enc(B) n x n (8-bit messages): "
                        "schoolbook, Strassen PC-MM (depths 1..5, schoolbook leaves) and Cussen on one GPU",
            "metric": "wall time per PC-MM and Cussen speed-up over Strassen and schoolbook", "unit": "ms",
            "rows": rows, "clocks": clk, "n_gpus": 1, "data": "synthetic (seeded)"}


def run_vector(args, dist):
    """Plaintext vector times ciphertext scalar (the paper's Sections 3.2 and
    4.2): a vector a of n t-bit entries times one ciphertext, giving n
    ciphertexts a_i Enc(b).  L products with independent ciphertext scalars
    and the same vector run as one PC-MM with A = a (n x 1) and Enc(B) 1 x L;
    the compression of a is shared, the table build of each scalar is the
    vector-scalar product.  Reports the device time per product (Cussen and
    schoolbook) and the point additions per second."""
    import torch

    from paper_2504_14497_gb300 import build, counts, inputs, pcmm

    build.build()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    pcmm.init(dist.local)
    seed = 2504144970 + 6
    L = int(args.vector_scalars)
    pr = inputs.pcmm_problem(seed, 1, 1, L, 1)
    tab = pcmm.keytable(pcmm.public_key(pr["sk"], device=dev), device=dev)
    ctB = pcmm.encrypt_table(tab, torch.from_numpy(pr["B"].reshape(-1)).to(dev),
                       pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev))
    cur = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            fn()
            e1.record(cur)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    rows = []
    for nv in (int(x) for x in args.vector_n.split(",")):
        out = torch.empty(48 * nv * L, dtype=torch.int32, device=dev)
        for w in (int(x) for x in args.vector_widths.split(",")):
            a_h = inputs.plaintext_matrix(seed, nv, 1, w)
            A = _host_plaintext(a_h).to(dev)
            ws = pcmm.workspace(nv, 1, L, w, 1, device=dev)
            ms = timed(lambda: pcmm.cussen(A, ctB, L, w, k=1, ws=ws, out=out))
            if pcmm.workspace_status(ws) != 0:
                raise RuntimeError(f"device status at n={nv} w={w}")
            del ws
            sb = timed(lambda: pcmm.schoolbook(A, ctB, L, w, out=out))
            ops = counts.point_ops(counts.cussen_counts(a_h, w, 1, L))
            rows.append({"n": nv, "t": w, "cussen_us_per_product": 1e3 * ms / L,
                         "schoolbook_us_per_product": 1e3 * sb / L, "speedup_vs_schoolbook": sb / ms,
                         "point_adds_per_s": ops / (ms / 1e3)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            torch.cuda.empty_cache()
        del out
        torch.cuda.empty_cache()
    return {"workload": f"vector x ciphertext scalar: a (n, t-bit) times {L} independent ciphertext scalars "
                        "as one PC-MM (A n x 1, Enc(B) 1 x L), 8-bit messages",
            "metric": "device time per vector-scalar product", "unit": "us", "scalars": L,
            "rows": rows, "n_gpus": 1, "data": "synthetic (seeded)"}


def run_sparse(args, dist):
    """The large product 1024 x 1024 x 256 with a sparse A (entries non-zero
    with probability rho, e.g. pruned weights): zero entries cost no point
    addition in the gather (their rank is skipped) and no table entry, so
    the time should follow the additions performed.  Per (w, rho): Cussen
    time (cost-model k, best of two after a warm-up), point additions
    performed and their rate, and the time relative to the dense matrix."""
    import torch

    from paper_2504_14497_gb300 import build, counts, inputs, pcmm

    build.build()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    pcmm.init(dist.local)
    m, n, l = 1024, 1024, 256
    pr = inputs.pcmm_problem(SEED, 1, n, l, 1)
    tab = pcmm.keytable(pcmm.public_key(pr["sk"], device=dev), device=dev)
    ctB = pcmm.encrypt_table(tab, torch.from_numpy(pr["B"].reshape(-1)).to(dev),
                       pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev))
    out = torch.empty(48 * m * l, dtype=torch.int32, device=dev)
    cur = torch.cuda.current_stream()

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            fn()
            e1.record(cur)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return best

    rows = []
    for w in (int(x) for x in args.sparse_widths.split(",")):
        k = pcmm.choose_k(m, n, l, w)
        ws = pcmm.workspace(m, n, l, w, k, device=dev)
        dense_ms = None
        for rho in (float(x) for x in args.sparse_densities.split(",")):
            A_h = inputs.sparse_plaintext(SEED + 11, m, n, w, rho)
            A = torch.from_numpy(A_h).to(dev)
            ms = timed(lambda: pcmm.cussen(A, ctB, l, w, k=k, ws=ws, out=out))
            if pcmm.workspace_status(ws) != 0:
                raise RuntimeError(f"device status at w={w} rho={rho}")
            # Per-kernel split of one more call (CUDA events around each launch).
            pcmm.profile_enable(64)
            pcmm.cussen(A, ctB, l, w, k=k, ws=ws, out=out)
            prof = pcmm.profile_read()
            pcmm.profile_enable(0)
            ops = counts.point_ops(counts.cussen_counts(A_h, w, k, l))
            dense_ms = ms if dense_ms is None else dense_ms
            rows.append({"w": w, "k": k, "density": rho, "nonzero_frac": float((A_h != 0).mean()),
                         "cussen_ms": ms, "table_ms": prof["table"][0], "gather_ms": prof["gather"][0],
                         "point_adds": ops, "point_adds_per_s": ops / (ms / 1e3),
                         "time_vs_first": ms / dense_ms})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        del ws
        torch.cuda.empty_cache()
    return {"workload": f"sparse: A {m}x{n} with entries non-zero with probability rho (uniform non-zero "
                        f"w-bit values) x Enc(B) {n}x{l} (8-bit messages), cost-model k",
            "metric": "Cussen PC-MM time per density", "unit": "ms", "rows": rows, "n_gpus": 1,
            "data": "synthetic (seeded)"}


def run_decrypt(args, dist):
    """Decryption of a PC-MM result by its key owner (Section 2.4): the
    1024 x 256 output of the large w = 8 product (262144 ciphertexts,
    messages up to n 255 255), decrypted on the GPU by baby-step giant-step
    with the default baby-step table (2^24 steps, four giant steps at most).
    Times the table build once and the decryption of every output over
    several steps (CUDA events), checks every message against the integer
    product A B, and times the CPU oracle's decryption on a bounded sample
    of the same ciphertexts."""
    import torch

    from paper_2504_14497_gb300 import build, counts, inputs, pcmm

    build.build()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    pcmm.init(dist.local)
    props = torch.cuda.get_device_properties(dev)
    m, n, l, w = 1024, 1024, 256, 8
    pr = inputs.pcmm_problem(SEED, m, n, l, w)
    tab = pcmm.keytable(pcmm.public_key(pr["sk"], device=dev), device=dev)
    ctB = pcmm.encrypt_table(tab, torch.from_numpy(pr["B"].reshape(-1)).to(dev),
                       pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev))
    A = torch.from_numpy(pr["A"]).to(dev)
    ct = pcmm.normalize(pcmm.cussen(A, ctB, l, w), m * l)
    del ctB
    torch.cuda.empty_cache()
    count, mmax = m * l, n * (2**w - 1) * 255
    cur = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    steps = pcmm.BabySteps.for_range(mmax, device=dev)
    e1.record(cur)
    e1.synchronize()
    build_ms = e0.elapsed_time(e1)
    out = torch.empty(count, dtype=torch.int64, device=dev)
    for _ in range(max(args.warmup, 1)):
        pcmm.decrypt(pr["sk"], ct, count, mmax, steps, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(dist.local)
    clocks.start()
    e0.record(cur)
    for _ in range(args.steps):
        pcmm.decrypt(pr["sk"], ct, count, mmax, steps, out=out)
    e1.record(cur)
    e1.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    AB = pr["A"].astype(np.int64) @ pr["B"].astype(np.int64)
    got = out.cpu().numpy().reshape(m, l)
    if not (got == AB).all():
        raise RuntimeError(f"decryption differs from A B at {int((got != AB).sum())} outputs")
    sk_int = int.from_bytes(np.asarray(pr["sk"], dtype="<u4").tobytes(), "little")
    prod = counts.decrypt_products(sk_int, AB, steps.baby)
    peak = measure_peaks(dev)["product"] * counts.IMAD_PER_PRODUCT   # measured, 2 IMAD per product
    imad_rate = count * prod * counts.IMAD_PER_PRODUCT / (ms / 1e3)
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle
        ns = 512
        aos = pcmm.planar_to_ct(pcmm.to_host_words(ct), count)[:ns]
        t0 = time.perf_counter()
        dec = oracle.decrypt(pr["sk"], aos, mmax)
        sec = time.perf_counter() - t0
        if not (dec == AB.reshape(-1)[:ns]).all():
            raise RuntimeError("oracle decryption differs from A B")
        cpu = {"value": ns / sec, "unit": "decryptions/s", "cores": oracle.threads(), "kind": "oracle",
               "sample": f"the first {ns} of the {count} output ciphertexts ({sec:.1f} s)"}
    return {"workload": f"decrypt: the {m}x{l} output of the w = {w} PC-MM {m}x{n} x Enc({n}x{l}), "
                        f"messages in [0, {mmax}], baby-step giant-step with {steps.baby} baby steps",
            "metric": "decryptions per second", "unit": "decryptions/s", "value": count / (ms / 1e3),
            "ms_per_step": ms, "steps": args.steps, "baby_table_build_ms": build_ms,
            "baby_table_bytes": steps.table.numel(), "verified_against_AB": True,
            "roofline": {"bound": "alu", "achieved": imad_rate / 1e12, "peak": peak / 1e12,
                         "unit": "T IMAD/s", "frac": imad_rate / peak,
                         "products_per_decryption": prod},
            "clocks": clk, "cpu_baseline": cpu, "n_gpus": 1, "data": "synthetic (seeded)"}


SERVING_MODELS = {"mlp_784": (256, 784), "mlp_256": (128, 256), "mlp_out": (10, 128)}


def run_serving(args, dist):
    """Encrypted linear-layer serving: Poisson arrivals over three resident
    models (4-bit weights), input batches of 1..64 encrypted column vectors
    (8-bit messages).  Continuous batching against one plain pcmm_cussen
    launch per request (plan rebuilt every time, one request at a time)."""
    import torch

    from paper_2504_14497_gb300 import counts, inputs, pcmm
    from paper_2504_14497_gb300.serving import GpuBackend, Request, Server

    rng = np.random.default_rng(SEED + 3)
    st = inputs.streams(SEED + 3)
    be = GpuBackend(f"cuda:{dist.local}", max_inflight=args.serving_inflight)
    dev = be.device
    weights = {nm: (st["A"].integers(0, 16, size=shape, dtype=np.uint8), 4, 0)
               for nm, shape in SERVING_MODELS.items()}
    srv_proto = dict(hbm_budget=40e9, max_inflight=args.serving_inflight, max_batch_cols=args.serving_cols)
    sk = inputs.uniform_scalars(st["sk"], (1,))[0]
    tab = pcmm.keytable(pcmm.public_key(sk, device=dev), device=dev)
    pool = []                                   # (model, l, ct) encrypted inputs
    for nm, (m, n) in SERVING_MODELS.items():
        for _ in range(6):
            l = int(rng.integers(1, 65))
            msg = st["B"].integers(0, 256, size=(n * l,), dtype=np.uint8)
            r = inputs.uniform_scalars(st["r"], (n * l,))
            ct = pcmm.encrypt_table(tab, torch.from_numpy(msg).to(dev),
                              pcmm.to_device_words(pcmm.scalars_to_planar(r), dev))
            pool.append((nm, l, ct))
    torch.cuda.synchronize()
    k_of = {nm: pcmm.choose_k(m, n, 256, 4) for nm, (m, n) in SERVING_MODELS.items()}
    ops_of = {}
    for nm, l, _ in pool:
        key = (nm, l)
        if key not in ops_of:
            ops_of[key] = counts.point_ops(counts.cussen_counts(weights[nm][0], 4, k_of[nm], l))

    def arrivals(rate):
        nreq = max(20, int(rate * args.seconds))
        t = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
        picks = rng.integers(0, len(pool), size=nreq)
        return [(float(ti), pool[int(p)]) for ti, p in zip(t, picks)]

    def summarise(lat, first, last, ops):
        lat = sorted(lat)
        pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
        span = max(last - first, 1e-9)
        return {"p50_ms": 1e3 * pct(0.5), "p99_ms": 1e3 * pct(0.99), "req_per_s": len(lat) / span,
                "point_adds_per_s": ops / span, "requests": len(lat)}

    rates = [float(x) for x in args.rates.split(",")]
    out_rates = []
    warm = Server(be, weights, **srv_proto)
    warm.run([Request(i, nm, ct, l, arrival=0.0) for i, (nm, l, ct) in enumerate(pool)])
    for rate in rates:
        arr = arrivals(rate)
        # Continuous batching.
        srv = Server(be, weights, **srv_proto)
        reqs = [Request(i, nm, ct, l, arrival=t) for i, (t, (nm, l, ct)) in enumerate(arr)]
        srv.run(reqs)
        ops = sum(ops_of[(r.model, r.l)] for r in srv.completed)
        cb = summarise([r.latency for r in srv.completed], min(r.arrival for r in reqs),
                       max(r.finish for r in srv.completed), ops)
        cb["batches"] = srv.stats()["batches"]
        # One plain launch per request, in arrival order.
        plain_A = {nm: torch.from_numpy(weights[nm][0]).to(dev) for nm in SERVING_MODELS}
        ws_cache = {}
        lat, t0 = [], time.perf_counter()
        for t, (nm, l, ct) in arr:
            while time.perf_counter() - t0 < t:
                pass
            m, n = SERVING_MODELS[nm]
            key = (nm, l)
            if key not in ws_cache:
                ws_cache[key] = pcmm.workspace(m, n, l, 4, k_of[nm], device=dev)
            jac = pcmm.cussen(plain_A[nm], ct, l, 4, k=k_of[nm], ws=ws_cache[key])
            pcmm.normalize(jac, m * l)
            torch.cuda.synchronize()
            lat.append(time.perf_counter() - t0 - t)
        last = time.perf_counter() - t0
        ops_p = sum(ops_of[(nm, l)] for _, (nm, l, _) in arr)
        pl = summarise(lat, arr[0][0], last, ops_p)
        out_rates.append({"rate": rate, "continuous_batching": cb, "one_launch_per_request": pl})
    return {"workload": "serving: Poisson encrypted linear layers over models "
                        + ", ".join(f"{m}x{n}" for m, n in SERVING_MODELS.values())
                        + " (4-bit weights), inputs of 1..64 encrypted columns, HBM budget 40 GB",
            "metric": "p50/p99 latency and requests/s per arrival rate", "n_gpus": 1,
            "rates": out_rates}


def main():
    args = parse()
    dist = Dist(args.gpus)
    try:
        if args.impl == "reference":
            out = run_reference(args, dist)
        elif args.workload == "serving":
            out = run_serving(args, dist)
        elif args.workload == "batched":
            out = run_batched(args, dist)
        elif args.workload == "sweep":
            out = run_sweep(args, dist)
        elif args.workload == "vector":
            out = run_vector(args, dist)
        elif args.workload == "decrypt":
            out = run_decrypt(args, dist)
        elif args.workload == "sparse":
            out = run_sparse(args, dist)
        elif args.workload == "strassen":
            out = run_strassen(args, dist)
        else:
            out = run_ours(args, dist)
        if dist.rank == 0 and out is not None:
            print(json.dumps(out), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
