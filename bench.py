#!/usr/bin/env python
"""LRAMM benchmark: effective TFLOP/s (2mnk / t) of Algorithm 3 on one GB300.

A step is one lramm_matmul call (RSVD of A and B, quantisation, E1/E2/E3
chain) with inputs resident in HBM.  Default workload: the rectangular
m = n = 32768, k = 4096 product (FP32 operands, sigma_i = (1+i)^-1.5,
r = 128, p = 16, q = 2, INT8 factors with per-row / per-column scales).
The L2 is flushed (256 MB write) before every timed step, outside the
step's event pair.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload W] [--variant int8|fp32|e4m3|...]
  python bench.py --impl reference ...   (the CPU oracle, timed on host cores)

Other workloads (--workload): lramm_512, lramm_4096, lramm_8192 run the
same step; rf_linear runs the range-finder form as a linear layer, one step =
forward C ~ X W plus the hand-written backward (dX, dW), effective
TFLOP/s = 6mnk / t (the dense layer's forward and backward GEMMs).

qsvd_4096 runs Algorithm 4 (quantised SVD of one matrix): a step is one
lramm_qsvd call producing the codes and scales of U~_k (d1) and V_k (d2);
the metric is input entries compressed per second.

Multi-GPU (torchrun): every rank runs an independent replica of the
workload; value = all ranks' work / max rank time (weak scaling).
"""
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

import workloads  # noqa: E402

METRIC = "effective TFLOP/s (2mnk/t) at stated rel. Frobenius error vs dense BF16 GEMM"
VARIANTS = {"int8": (1, 1, 1), "fp32": (0, 0, 0), "e4m3": (3, 3, 3), "884": (1, 1, 2),
            "lead64_mxfp4": (1, 1, 4), "lead64_int4": (1, 1, 2)}
DTYPES = {"int8": "f32+int8", "fp32": "f32", "e4m3": "f32+e4m3", "884": "f32+int8+int4",
          "lead64_mxfp4": "int8+mxfp4", "lead64_int4": "int8+int4"}
# E3 lead / tail split (lead rank directions, lead precision, residual terms)
LEADS = {"lead64_mxfp4": (64, 1, 2), "lead64_int4": (64, 1, 2)}
FLUSH_BYTES = 256 << 20
QSVD_METRIC = "quantised-SVD compression throughput (Algorithm 4): input entries per second"
# Algorithm 4's bit widths (d1 for U~_k, d2 for V_k) per variant
QSVD_BITS = {"int8": (1, 1), "884": (1, 2), "e4m3": (3, 3), "lead64_int4": (1, 2)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ ranks
def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank gets it); ms unchanged without a process group."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(world, flops_per_step, steps, max_ms):
    """Whole-job throughput: every rank's work over the slowest rank's time (weak scaling)."""
    return world * flops_per_step * steps / (max_ms * 1e-3) / 1e12


# ------------------------------------------------------------------ roofline
def kernel_work(kind, cfg, l, variant):
    """Algorithmic (bytes, flops) of ONE launch of a kernel kind on this workload.

    sketch: one product of an operand X (rows x cols) with an l-column
      matrix; bytes = X once + the l-column input + the l-column output.
    e3: the m x n output written once (FP32) plus both code operands read;
      flops 2 m n r.
    """
    m, n, k, r = cfg["m"], cfg["n"], cfg["k"], cfg["r"]
    xb = 2 if cfg["dtype"] == "bf16" else 4
    if kind == "sketch":
        return (m * k * xb + (m + k) * l * 4, 2.0 * m * k * l)
    if kind == "e3":
        cb = 2 if VARIANTS[variant][2] == 1 else (4 if VARIANTS[variant][2] == 0 else 1)
        return (4 * m * n + (m + n) * r * cb, 2.0 * m * n * r)
    if kind == "gram":
        return (4 * m * l, 2.0 * m * l * l)
    if kind == "trsm":
        return (8 * m * l, 1.0 * m * l * l)
    return (None, None)


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# the ncu captures summarised under profiles/, per workload, for the kernels
# as they are in this tree; None where no capture of the current kernel
# exists.  lramm_32768: the sketch's mean over the 12 launches of one call
# (profiles/sketch_tc_lramm_32768.md, a one-pass capture at full size); E3
# scaled by 4 from the 16384 x 16384 capture (profiles/e3_qgemm_tcp_lramm_32768.md:
# the traffic is the output write, proportional to m n).
MEASURED_TRAFFIC = {
    "lramm_32768": {"sketch": 547600000 + 500000, "e3": 4 * (1012497000 + 8663040)},
    "lramm_4096": {"svd": 350208},   # the M-only Jacobi (profiles/jacobi_monly_lramm_4096.md)
}


def measured_traffic(workload, kind):
    return MEASURED_TRAFFIC.get(workload, {}).get(kind)


def jacobi_work(l, sweeps, with_v=True):
    """Algorithmic FP32 flops of one launch of the one-sided Jacobi SVD (one
    operand per launch: the two operands' SVDs run on two streams; `sweeps`
    lists both, the result is their mean): per sweep every one of the
    l(l-1)/2 column pairs forms three inner products of length l (6 l flops)
    and rotates its two columns of M and of V (4 vectors x 3 l flops) -- 18 l
    flops per pair; 12 l in the M-only form (no V accumulated)."""
    per_pair = 18.0 if with_v else 12.0
    return sum(s * l * (l - 1) / 2 * per_pair * l for s in sweeps) / max(len(sweeps), 1)


def m_only_svd(variant, l):
    """Quantised chains (a quantised E3, or a lead / tail split) of l <= 544
    take the M-only small SVD inside lramm_matmul."""
    return (VARIANTS[variant][2] != 0 or variant in LEADS) and l <= 544


def fp32_alu_peak_tflops(sm_mhz):
    """152 SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_step(A, B, cfg, prec, lead=None, rows=None):
    """Seconds of one oracle LRAMM step on A, B (FP32 numpy).

    rows: a sorted sample of A's row indices, for outputs too large to form
    on the host: the randomized SVDs of both operands and E1, E2 run in full,
    E3 (whose cost is proportional to the rows of U~; per-row scales make
    each output row independent of the others) on the sampled rows only,
    its time scaled by m / len(rows)."""
    import oracle
    r, p, q = cfg["r"], cfg["p"], cfg["q"]
    t0 = time.perf_counter()
    if rows is None:
        if lead:
            fac = oracle.lramm.factors(A, B, r, p, q, workloads.SEED_SKETCH)
            oracle.mixed.chain_lead_tail(*fac, prec, min(lead[0], r), lead[1], lead[2])
        else:
            oracle.lramm.lramm(A, B, r, p, q, workloads.SEED_SKETCH, prec)
        return time.perf_counter() - t0
    Ut, V, W, Zt = oracle.lramm.factors(A, B, r, p, q, workloads.SEED_SKETCH)
    E1 = oracle.mixed.qm_any(np.asarray(V, np.float32).T, W, prec[0], oracle.quant.SCALE_ROWCOL)
    E2 = oracle.mixed.qm_any(E1, Zt, prec[1], oracle.quant.SCALE_ROWCOL)
    t1 = time.perf_counter()
    Us = Ut[rows]
    if lead:
        oracle.mixed.e3_lead_tail(Us, E2, prec[2], min(lead[0], r), lead[1], lead[2])
    else:
        oracle.mixed.qm_any(Us, E2, prec[2], oracle.quant.SCALE_ROWCOL)
    t2 = time.perf_counter()
    return (t1 - t0) + (t2 - t1) * A.shape[0] / len(rows)


# outputs with more entries than this are formed on a seeded row sample
# (the error against the FP64 product and the oracle's E3)
SAMPLE_ENTRIES = 1 << 28
SAMPLE_ROWS = 2048


def sample_rows(m, n):
    """The seeded row sample of an m x n output (None: all rows)."""
    if m * n <= SAMPLE_ENTRIES:
        return None
    return np.sort(np.random.default_rng(5).choice(m, SAMPLE_ROWS, replace=False))


def cpu_sample(name):
    """A bounded stand-in of the workload for the CPU oracle: every size
    halved (r and p too) until the problem has at most 4096^3 multiply-adds,
    for when the full-shape oracle step would not fit the run's time."""
    c = dict(workloads.CONFIGS[name])
    sc = (c["m"], c["n"], c["k"])
    while sc[0] * sc[1] * sc[2] > 4096 ** 3:
        sc = tuple(max(256, s // 2) for s in sc)
        c["r"] = max(16, c["r"] // 2)
        c["p"] = max(4, c["p"] // 2)
    A, B = workloads.operands(name, scale=sc)
    c["m"], c["n"], c["k"] = sc
    return A.astype(np.float32), B.astype(np.float32), c


def cpu_rf_sample():
    """A bounded stand-in of the linear-layer workload for the CPU oracle:
    every size divided by 4 (X 4096 x 1024, W 1024 x 2752, r = 96, p = 4)."""
    c = dict(workloads.CONFIGS["rf_linear"])
    c["m"], c["n"], c["k"], c["r"], c["p"] = c["m"] // 4, c["n"] // 4, c["k"] // 4, c["r"] // 4, c["p"] // 4
    X, W = workloads.operands("rf_linear", scale=(c["m"], c["n"], c["k"]))
    G = np.random.default_rng(17).standard_normal((c["m"], c["n"])).astype(np.float32)
    return X.astype(np.float32), W.astype(np.float32), G, c


def cpu_rf_step(X, W, G, c, prec):
    import oracle
    t0 = time.perf_counter()
    oracle.rf.rf_forward(X, W, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, prec=prec)
    oracle.rf.rf_backward(X, W, G, c["r"], c["p"], c["q"], workloads.SEED_SKETCH)
    return time.perf_counter() - t0


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    """--impl reference: the oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prec = VARIANTS[args.variant]
    if args.workload == "qsvd_4096":
        return run_reference_qsvd(args)
    if args.workload == "rf_linear":
        X, W, G, c = cpu_rf_sample()
        flops = 6.0 * c["m"] * c["n"] * c["k"]
        step = lambda: cpu_rf_step(X, W, G, c, prec[2])  # noqa: E731
        what = "oracle range-finder forward + backward"
    else:
        # the full workload, E3 on a seeded row sample when the output is
        # too large for the host (see cpu_oracle_step); one untimed probe step
        # checks that the run (warm-up + timed steps) stays within about two
        # and a half minutes of host work, else every size of a stand-in is
        # halved while a step would take longer
        lead = LEADS.get(args.variant)
        c = dict(workloads.CONFIGS[args.workload])
        budget = 150.0 / max(1, args.steps + args.warmup)
        A, B = workloads.operands(args.workload)
        A, B = A.astype(np.float32), B.astype(np.float32)
        rows = sample_rows(c["m"], c["n"])
        w0 = time.perf_counter()
        cpu_oracle_step(A, B, c, prec, lead, rows)
        if time.perf_counter() - w0 > budget:
            rows = None
            A, B, c = cpu_sample(args.workload)
            t_probe = cpu_oracle_step(A, B, c, prec, lead)
            while t_probe > budget and min(c["m"], c["n"], c["k"]) > 512:
                sc = tuple(max(256, x // 2) for x in (c["m"], c["n"], c["k"]))
                c["r"], c["p"] = max(16, c["r"] // 2), max(4, c["p"] // 2)
                A, B = workloads.operands(args.workload, scale=sc)
                A, B = A.astype(np.float32), B.astype(np.float32)
                c["m"], c["n"], c["k"] = sc
                t_probe = cpu_oracle_step(A, B, c, prec, lead)
        flops = 2.0 * c["m"] * c["n"] * c["k"]
        step = lambda: cpu_oracle_step(A, B, c, prec, lead, rows)  # noqa: E731
        what = "oracle LRAMM" + ("" if rows is None else
                                 " (randomized SVDs, E1, E2 in full; E3 on %d seeded rows, time scaled by m/%d)"
                                 % (len(rows), len(rows)))
    for _ in range(args.warmup):
        step()
    ts = [step() for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    v = flops / t / 1e12
    sample = "%s at m=%d n=%d k=%d r=%d p=%d q=%d per step" % (what, c["m"], c["n"], c["k"], c["r"], c["p"], c["q"])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "variant": args.variant, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def qsvd_cpu_sample(full=False):
    """The quantised-SVD workload for the CPU oracle: the full 4096 x 4096
    matrix (full=True), else a bounded stand-in with the same spectrum rule
    at 2048 x 2048, r = 128, p = 8 (the reference arm's per-step sample)."""
    c = dict(workloads.CONFIGS["qsvd_4096"])
    if not full:
        c["m"] = c["n"] = c["k"] = 2048
        c["r"], c["p"] = 128, 8
    A, _ = workloads.operands("qsvd_4096", scale=(c["m"], c["n"], c["k"]))
    return A.astype(np.float32), c


def cpu_qsvd_step(A, c, bits):
    import oracle
    t0 = time.perf_counter()
    oracle.qsvd.qsvd(A, c["r"], c["p"], c["q"], workloads.SEED_SKETCH, 0, bits[0], bits[1])
    return time.perf_counter() - t0


def run_reference_qsvd(args):
    bits = QSVD_BITS[args.variant]
    A, c = qsvd_cpu_sample()
    for _ in range(args.warmup):
        cpu_qsvd_step(A, c, bits)
    ts = [cpu_qsvd_step(A, c, bits) for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    v = c["m"] * c["k"] / t / 1e9
    sample = "oracle Algorithm 4 at %d x %d, r=%d p=%d q=%d per step" % (c["m"], c["k"], c["r"], c["p"], c["q"])
    line = {"impl": "reference", "metric": QSVD_METRIC, "value": v, "unit": "Gentries/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "variant": args.variant, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "Gentries/s", "cores": cores_used(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "Gentries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def run_lramm(args):
    import torch

    import paper_2405_16917_gb300 as L

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    L.load()
    cfg = dict(workloads.CONFIGS[args.workload])
    if args.mn_div > 1:   # a reduced instance: m and n divided, k, r, p, q kept
        cfg["m"], cfg["n"] = cfg["m"] // args.mn_div, cfg["n"] // args.mn_div
    m, n, k, r, p, q = cfg["m"], cfg["n"], cfg["k"], cfg["r"], cfg["p"], cfg["q"]
    l = r + p
    prec = VARIANTS[args.variant]
    A, B = workloads.device_operands(args.workload, dev, sizes=(m, n, k))
    a_type = L.BF16 if A.dtype == torch.bfloat16 else L.F32
    sketch_name = args.sketch or ("fp32" if args.variant == "fp32" else "tf32")
    sketch = {"tf32": L.SKETCH_TF32, "fp32": L.SKETCH_F32, "e4m3": L.SKETCH_E4M3}[sketch_name]
    lead = LEADS.get(args.variant, (0, 1, 0))
    # the timed steps run an uninstrumented plan; a second, instrumented plan
    # (CUDA events around every kernel) gives the per-kind breakdown
    plan = L.Plan(m, n, k, r, p, q, seed=workloads.SEED_SKETCH, prec=prec, a_type=a_type, b_type=a_type,
                  sketch=sketch, lead=lead[0], lead_prec=lead[1], lead_split=lead[2], graph=True)
    tplan = L.Plan(m, n, k, r, p, q, seed=workloads.SEED_SKETCH, prec=prec, a_type=a_type, b_type=a_type,
                   sketch=sketch, timing=True, lead=lead[0], lead_prec=lead[1], lead_split=lead[2])
    ws = plan.workspace(dev)
    D = torch.empty((m, n), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # a non-default stream: the plan captures its call into a CUDA graph there
    # (the first warm-up step) and replays it afterwards
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    for _ in range(max(args.warmup, 0)):
        L.matmul(plan, A, B, out=D, ws=ws)
    info = L.info_read(ws, 3)
    st = L.status_read(ws)
    if st != 0:
        raise RuntimeError("device status %d after warm-up" % st)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kinds = {}
    gpu_id = local
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    n_launch0 = L.launch_count()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        L.matmul(plan, A, B, out=D, ws=ws)
        ends[i].record(stream)
    n_launch = L.launch_count() - n_launch0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dist, dev)
    ms_step = total_ms / args.steps
    flops = 2.0 * m * n * k
    value = whole_job_tflops(world, flops, args.steps, total_ms)
    st = L.status_read(ws)

    # per-kind device time (instrumented plan, outside the timed region)
    nbd = min(args.steps, 5)
    for i in range(nbd):
        flush.zero_()
        L.matmul(tplan, A, B, out=D, ws=ws)
        for kname, (ms, cnt) in tplan.timing().items():
            a = kinds.setdefault(kname, [0.0, 0])
            a[0] += ms
            a[1] += cnt

    # accuracy of this variant and of the comparators (outside the timed region);
    # outputs above 2^28 entries are compared on a seeded sample of 2048 rows
    rows_np = sample_rows(m, n)
    rows = None if rows_np is None else torch.from_numpy(rows_np).to(dev)
    Asub = A if rows is None else A[rows]
    exact = Asub.double() @ B.double()
    nrm = exact.norm().item()

    def rel_err(X):
        Xs = X if rows is None else X[rows]
        return ((Xs.double() - exact).norm() / nrm).item()

    err = rel_err(D)

    def timed(fn, reps=3):
        for _ in range(2):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    A16, B16 = A.to(torch.bfloat16), B.to(torch.bfloat16)
    Cb = torch.empty((m, n), dtype=torch.bfloat16, device=dev)
    t_bf16 = timed(lambda: torch.matmul(A16, B16, out=Cb))
    err_bf16 = rel_err(Cb)
    # the paper's direct quantised comparators DQ8 / DQ4 (Algorithm 2 on the full operands)
    Af, Bf = A.float(), B.float()
    Dq = torch.empty((m, n), dtype=torch.float32, device=dev)
    dq = {}
    for name, pq in (("dq8", 1), ("dq4", 2)):
        wsq = torch.empty(L.load().lramm_dq_ws_bytes(pq, m, n, k), dtype=torch.uint8, device=dev)
        t_dq = timed(lambda: L.dq_matmul(Af, Bf, prec=pq, out=Dq, ws=wsq))
        dq[name] = {"tflops": flops / (t_dq * 1e-3) / 1e12, "ms": t_dq, "rel_fro_err_vs_fp64_exact": rel_err(Dq)}
        del wsq
    del Af, Bf, Dq
    plain = L.Plan(m, n, k, r, p, q, seed=workloads.SEED_SKETCH, prec=(0, 0, 0), a_type=a_type, b_type=a_type)
    Dp = torch.empty_like(D)
    t_plain = timed(lambda: L.matmul(plan=plain, A=A, B=B, out=Dp, ws=ws), reps=2)
    err_plain = rel_err(Dp)
    del exact

    # end to end through the public API with host buffers: every step copies
    # its A and B from pinned host memory to the device, runs lramm_matmul and
    # reads its D back to pinned host memory.  Two buffer sets (and two plans
    # sharing one workspace, so that each keeps its captured graph) pipeline
    # the steps: step i+1's host-to-device copies and step i's device-to-host
    # copy run on their own streams beside the compute stream.
    Ah, Bh = A.cpu().pin_memory(), B.cpu().pin_memory()
    Dh = torch.empty((m, n), dtype=torch.float32).pin_memory()
    del Dp
    Ad = [torch.empty_like(A) for _ in range(2)]
    Bd = [torch.empty_like(B) for _ in range(2)]
    Dd = [D, torch.empty_like(D)]
    plans = [plan, L.Plan(m, n, k, r, p, q, seed=workloads.SEED_SKETCH, prec=prec, a_type=a_type, b_type=a_type,
                          sketch=sketch, lead=lead[0], lead_prec=lead[1], lead_split=lead[2], graph=True)]
    s_h2d, s_d2h = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]     # inputs of buffer b on the device
    ev_done = [torch.cuda.Event() for _ in range(2)]   # step on buffer b computed
    ev_out = [torch.cuda.Event() for _ in range(2)]    # D of buffer b read back
    for e in ev_done + ev_out:
        e.record(stream)

    def e2e_step(i):
        b = i % 2
        s_h2d.wait_event(ev_done[b])             # buffer b's inputs no longer read
        with torch.cuda.stream(s_h2d):
            Ad[b].copy_(Ah, non_blocking=True)
            Bd[b].copy_(Bh, non_blocking=True)
        ev_in[b].record(s_h2d)
        stream.wait_event(ev_in[b])
        stream.wait_event(ev_out[b])              # buffer b's D read back
        L.matmul(plans[b], Ad[b], Bd[b], out=Dd[b], ws=ws)
        ev_done[b].record(stream)
        s_d2h.wait_event(ev_done[b])
        with torch.cuda.stream(s_d2h):
            Dh.copy_(Dd[b], non_blocking=True)
        ev_out[b].record(s_d2h)

    e2e_steps = max(4, min(args.steps, 8))
    for i in range(2):
        e2e_step(i)
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    s_h2d.wait_event(ea)
    s_d2h.wait_event(ea)
    for i in range(e2e_steps):
        e2e_step(i)
    for st_ in (s_h2d, s_d2h):
        e_ = torch.cuda.Event()
        e_.record(st_)
        stream.wait_event(e_)
    eb.record(stream)
    eb.synchronize()
    e2e_ms = ea.elapsed_time(eb) / e2e_steps
    e2e_val = world * flops / (e2e_ms * 1e-3) / 1e12
    e2e_ok = L.status_read(ws) == 0 and bool(torch.equal(Dh[:4], Dd[(e2e_steps - 1) % 2][:4].cpu()))
    del Ad, Bd, Dd

    # roofline of the dominant kernel kind (largest device time in the timed steps)
    pk, peak_src = peaks()
    dom = max(kinds.items(), key=lambda kv: kv[1][0])
    dname, (dms, dcnt) = dom
    avg_s = dms / dcnt * 1e-3
    nbytes, nflops = kernel_work(dname, cfg, l, args.variant)
    sm_mhz = clk.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    if dname == "sketch" and sketch_name == "tf32":
        # tcgen05 products streaming X once: bound by HBM bandwidth
        roof = {"bound": "hbm", "achieved": nbytes / avg_s / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "kernel": dname, "launches_per_step": dcnt / nbd, "avg_launch_ms": avg_s * 1e3,
                "peak_source": peak_src + " hbm_gbs", "traffic": None, "algorithmic_bytes_per_launch": nbytes}
        roof["frac"] = roof["achieved"] / roof["peak"]
    elif dname in ("sketch", "e3", "gram", "trsm", "e1", "e2") and nflops is not None and sketch_name != "e4m3":
        # these kernels are FP32 SIMT in this version: bound by FP32 FMA issue
        roof = {"bound": "alu", "achieved": nflops / avg_s / 1e12,
                "peak": fp32_alu_peak_tflops(pk.get("sm_max_mhz", 2070.0)), "unit": "TFLOP/s",
                "kernel": dname, "launches_per_step": dcnt / nbd,
                "avg_launch_ms": avg_s * 1e3, "peak_source": "derived: 152 SM x 128 FP32 FMA x 2 x sm_max_mhz"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["traffic"] = None
        roof["algorithmic_bytes_per_launch"] = nbytes
    elif dname == "svd":
        # latency-bound: l sequential rounds per sweep; reported against the FP32 ALU roof
        mo = m_only_svd(args.variant, l)
        jf = jacobi_work(l, [int(x) for x in info[1:3] if int(x) > 0], with_v=not mo)
        roof = {"bound": "alu", "achieved": jf / avg_s / 1e12,
                "peak": fp32_alu_peak_tflops(pk.get("sm_max_mhz", 2070.0)), "unit": "TFLOP/s",
                "kernel": dname, "launches_per_step": dcnt / nbd, "avg_launch_ms": avg_s * 1e3,
                "peak_source": "derived: 152 SM x 128 FP32 FMA x 2 x sm_max_mhz",
                "traffic": measured_traffic(args.workload, "svd") if mo else None,
                "algorithmic_flops_per_launch": jf,
                "note": "one-sided Jacobi, sequential rounds of column-pair rotations on a 16-CTA cluster "
                        "(one launch per operand, the two on concurrent streams)"
                        + ("; M-only form (no V accumulated): 12 l flops per pair" if mo else "")}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        roof = {"bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                "kernel": dname, "launches_per_step": dcnt / nbd, "avg_launch_ms": avg_s * 1e3,
                "note": "latency-bound small factorisation; no algorithmic roof"}
    # the bandwidth-bound kernels, each against its own roof (same definitions)
    kroofs = {}
    for kn in ("sketch", "e3"):
        if kn not in kinds:
            continue
        kms, kc = kinds[kn]
        ks = kms / kc * 1e-3
        kb, kf = kernel_work(kn, cfg, l, args.variant)
        if kn == "sketch" and sketch_name not in ("tf32",):
            continue
        kroofs[kn] = {"bound": "hbm", "achieved": kb / ks / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                      "frac": kb / ks / 1e9 / pk["hbm_gbs"], "avg_launch_ms": ks * 1e3,
                      "launches_per_step": kc / nbd, "algorithmic_bytes_per_launch": kb,
                      "traffic": measured_traffic(args.workload, kn)}

    # CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the workload's own operands at full size (FP32 on the host; BF16
        # operands widen exactly), E3 on the error's row sample when the
        # output is too large for the host
        Ac, Bc = A.float().cpu().numpy(), B.float().cpu().numpy()
        t_cpu = cpu_oracle_step(Ac, Bc, cfg, prec, LEADS.get(args.variant), rows_np)
        del Ac, Bc
        cpu = {"value": flops / t_cpu / 1e12, "unit": "TFLOP/s", "cores": cores_used(), "kind": "oracle",
               "sample": "one oracle LRAMM step at m=%d n=%d k=%d r=%d p=%d q=%d%s, %.1f s"
                         % (m, n, k, r, p, q,
                            "" if rows_np is None else
                            " (randomized SVDs, E1, E2 in full; E3 on the %d sampled rows, its time scaled by "
                            "m/%d)" % (len(rows_np), len(rows_np)), t_cpu)}

    launches = n_launch
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPES[args.variant], "data": "synthetic",
            "config": {"workload": args.workload, "m": m, "n": n, "k": k, "r": r, "p": p, "q": q,
                       "variant": args.variant, "operands": cfg["dtype"], "spectrum": cfg["spectrum"],
                       "lead": {"directions": lead[0], "prec": lead[1], "residual_terms": lead[2]} if lead[0] else None,
                       "sketch": sketch_name, "scale": "rowcol", "cuda_graph": True,
                       "jacobi_sweeps": info[1:3], "l2": "flushed: 256 MB write before each step",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "rel_fro_err_vs_fp64_exact": err,
                       "err_rows": "all" if rows is None else "%d sampled rows (seed 5)" % SAMPLE_ROWS,
                       "dense_bf16_gemm": {"tflops": flops / (t_bf16 * 1e-3) / 1e12, "ms": t_bf16,
                                           "rel_fro_err_vs_fp64_exact": err_bf16},
                       "plain_lramm_fp32": {"tflops": flops / (t_plain * 1e-3) / 1e12, "ms": t_plain,
                                            "rel_fro_err_vs_fp64_exact": err_plain},
                       "direct_quantised": dq,
                       "device_status": st},
            "breakdown_ms_per_step": {kn: round(v[0] / nbd, 4) for kn, v in
                                      sorted(kinds.items(), key=lambda kv: -kv[1][0])},
            "breakdown_note": "CUDA events around every kernel of %d separate steps; both operands' streams "
                              "summed" % nbd,
            "roofline": roof,
            "kernel_rooflines": kroofs,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": A.numel() * A.element_size() + B.numel() * B.element_size(),
                    "d2h_bytes_per_step": D.numel() * D.element_size(), "steps": e2e_steps,
                    "pipelined": "two buffer sets: step i+1's host-to-device copies and step i's device-to-host "
                                 "copy overlap the compute stream", "result_checked": e2e_ok},
            "gpu_launches": launches,
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons"), "samples": clk.get("samples")},
            "peaks": peak_src,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ range-finder form
def run_rf(args):
    """The linear-layer workload: C ~ X W in the range-finder form, forward
    plus the hand-written backward (dX, dW) per step."""
    import torch

    import paper_2405_16917_gb300 as L

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    L.load()
    cfg = workloads.CONFIGS["rf_linear"]
    m, n, k, r, p, q = cfg["m"], cfg["n"], cfg["k"], cfg["r"], cfg["p"], cfg["q"]
    l = r + p
    prec = VARIANTS[args.variant][2]
    X32, W = workloads.device_operands("rf_linear", dev, dtype=torch.float32)
    X = X32.to(torch.bfloat16).contiguous()
    del X32
    g = torch.Generator(device=dev)
    g.manual_seed(17)
    G = torch.randn((m, n), generator=g, device=dev, dtype=torch.float32)
    sketch_name = args.sketch or ("fp32" if args.variant == "fp32" else "tf32")
    sketch = {"tf32": L.SKETCH_TF32, "fp32": L.SKETCH_F32, "e4m3": L.SKETCH_E4M3}[sketch_name]
    plan = L.Plan(m, n, k, r, p, q, seed=workloads.SEED_SKETCH, prec=(0, 0, prec), a_type=L.BF16, b_type=L.F32,
                  sketch=sketch)
    tplan = L.Plan(m, n, k, r, p, q, seed=workloads.SEED_SKETCH, prec=(0, 0, prec), a_type=L.BF16, b_type=L.F32,
                   sketch=sketch, timing=True)
    ws = plan.workspace(dev)
    C = torch.empty((m, n), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    kinds = {}

    def collect():
        for kname, (ms, cnt) in tplan.timing().items():
            a = kinds.setdefault(kname, [0.0, 0])
            a[0] += ms
            a[1] += cnt

    def step(record):
        pl = tplan if record else plan
        out = L.rf_forward(pl, X, W, C=C, ws=ws)
        if record:
            collect()
        grads = L.rf_backward(pl, X, W, G, ws=ws)
        if record:
            collect()
        return out, grads

    for _ in range(max(args.warmup, 0)):
        step(False)
    st = L.status_read(ws)
    if st != 0:
        raise RuntimeError("device status %d after warm-up" % st)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    gpu_id = local
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    n_launch0 = L.launch_count()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        _, (dX, dW) = step(False)
        ends[i].record(stream)
    n_launch = L.launch_count() - n_launch0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    total_ms = max_over_ranks(total_ms, dist, dev)
    ms_step = total_ms / args.steps
    flops = 6.0 * m * n * k
    value = whole_job_tflops(world, flops, args.steps, total_ms)
    st = L.status_read(ws)
    nbd = min(args.steps, 3)   # instrumented steps for the per-kind breakdown (outside the timed region)
    for _ in range(nbd):
        flush.zero_()
        step(True)

    # accuracy (outside the timed region): forward against X W, gradients
    # against the dense layer's G W^T and X^T G, all in FP64 on the device
    Xd, Wd, Gd = X.double(), W.double(), G.double()
    ex_c = Xd @ Wd
    err_c = ((C.double() - ex_c).norm() / ex_c.norm()).item()
    del ex_c
    ex_dx = Gd @ Wd.T
    err_dx = ((dX.double() - ex_dx).norm() / ex_dx.norm()).item()
    del ex_dx
    ex_dw = Xd.T @ Gd
    err_dw = ((dW.double() - ex_dw).norm() / ex_dw.norm()).item()
    del ex_dw, Xd, Wd, Gd
    torch.cuda.empty_cache()

    def timed(fn, reps=3):
        for _ in range(2):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    W16, G16 = W.to(torch.bfloat16), G.to(torch.bfloat16)
    Cb = torch.empty((m, n), dtype=torch.bfloat16, device=dev)
    dXb = torch.empty((m, k), dtype=torch.bfloat16, device=dev)
    dWb = torch.empty((k, n), dtype=torch.bfloat16, device=dev)

    def dense():
        torch.matmul(X, W16, out=Cb)
        torch.matmul(G16, W16.T, out=dXb)
        torch.matmul(X.T, G16, out=dWb)

    t_bf16 = timed(dense)
    del W16, G16, Cb, dXb, dWb

    # end to end with host buffers: X, W, G in from pinned memory, C, dX, dW out
    Xh, Wh, Gh = X.cpu().pin_memory(), W.cpu().pin_memory(), G.cpu().pin_memory()
    Ch = torch.empty((m, n), dtype=torch.float32).pin_memory()
    dXh = torch.empty((m, k), dtype=torch.float32).pin_memory()
    dWh = torch.empty((k, n), dtype=torch.float32).pin_memory()
    Xe, We, Ge = torch.empty_like(X), torch.empty_like(W), torch.empty_like(G)

    def e2e_step():
        Xe.copy_(Xh, non_blocking=True)
        We.copy_(Wh, non_blocking=True)
        Ge.copy_(Gh, non_blocking=True)
        L.rf_forward(plan, Xe, We, C=C, ws=ws)
        a, b = L.rf_backward(plan, Xe, We, Ge, ws=ws)
        Ch.copy_(C, non_blocking=True)
        dXh.copy_(a, non_blocking=True)
        dWh.copy_(b, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e2e_steps = max(2, min(args.steps, 5))
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    eb.record(stream)
    eb.synchronize()
    e2e_ms = ea.elapsed_time(eb) / e2e_steps
    e2e_val = world * flops / (e2e_ms * 1e-3) / 1e12

    pk, peak_src = peaks()
    dname, (dms, dcnt) = max(kinds.items(), key=lambda kv: kv[1][0])
    avg_s = dms / dcnt * 1e-3
    roof = {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
            "kernel": dname, "launches_per_step": dcnt / nbd, "avg_launch_ms": avg_s * 1e3,
            "note": "no per-launch algorithmic figure for this kind in the range-finder form"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Xc, Wc, Gc, cs = cpu_rf_sample()
        t_cpu = cpu_rf_step(Xc, Wc, Gc, cs, prec)
        cpu = {"value": 6.0 * cs["m"] * cs["n"] * cs["k"] / t_cpu / 1e12, "unit": "TFLOP/s",
               "cores": cores_used(), "kind": "oracle",
               "sample": "one oracle range-finder forward + backward at m=%d n=%d k=%d r=%d p=%d q=%d, %.1f s"
                         % (cs["m"], cs["n"], cs["k"], cs["r"], cs["p"], cs["q"], t_cpu)}
    launches = n_launch
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16+f32+" + ("e4m3" if prec == 3 else ("int8" if prec == 1 else "f32")),
            "data": "synthetic",
            "config": {"workload": "rf_linear", "m": m, "n": n, "k": k, "r": r, "p": p, "q": q,
                       "variant": args.variant, "form": "range-finder, forward + backward",
                       "flops_per_step": "6mnk (dense forward 2mnk + backward dX, dW 4mnk)",
                       "sketch": sketch_name, "l2": "flushed: 256 MB write before each step",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "rel_fro_err_forward_vs_fp64_xw": err_c,
                       "rel_fro_err_dx_vs_fp64_dense": err_dx, "rel_fro_err_dw_vs_fp64_dense": err_dw,
                       "dense_bf16_fwd_bwd": {"tflops": flops / (t_bf16 * 1e-3) / 1e12, "ms": t_bf16},
                       "device_status": st},
            "breakdown_ms_per_step": {kn: round(v[0] / nbd, 4) for kn, v in
                                      sorted(kinds.items(), key=lambda kv: -kv[1][0])},
            "breakdown_note": "CUDA events around every kernel of %d separate steps" % nbd,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": X.numel() * X.element_size() + W.numel() * W.element_size()
                    + G.numel() * G.element_size(),
                    "d2h_bytes_per_step": 4 * (m * n + m * k + k * n)},
            "gpu_launches": launches,
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons"), "samples": clk.get("samples")},
            "peaks": peak_src,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ Algorithm 4
def run_qsvd(args):
    """Quantised SVD of one matrix: one lramm_qsvd call per step (codes and
    scales of U~_k and V_k); the approximation deq(U~') deq(V')^T timed beside it."""
    import torch

    import paper_2405_16917_gb300 as L

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    lib = L.load()
    cfg = workloads.CONFIGS["qsvd_4096"]
    m, k, r, p, q = cfg["m"], cfg["k"], cfg["r"], cfg["p"], cfg["q"]
    l = r + p
    if args.variant not in QSVD_BITS:
        raise SystemExit("qsvd_4096: variant must be one of %s" % sorted(QSVD_BITS))
    pu, pv = QSVD_BITS[args.variant]
    A, _ = workloads.device_operands("qsvd_4096", dev)
    sketch_name = args.sketch or "tf32"
    sketch = {"tf32": L.SKETCH_TF32, "fp32": L.SKETCH_F32, "e4m3": L.SKETCH_E4M3}[sketch_name]
    plan = L.Plan(m, k, k, r, p, q, seed=workloads.SEED_SKETCH, sketch=sketch)
    tplan = L.Plan(m, k, k, r, p, q, seed=workloads.SEED_SKETCH, sketch=sketch, timing=True)
    ws = torch.empty(lib.lramm_qsvd_ws_bytes(plan.handle, 0, pu, pv), dtype=torch.uint8, device=dev)
    ldq = -(-r // 32) * 32
    Uc = torch.empty((m, ldq), dtype=L.code_dtype(pu), device=dev)
    Vc = torch.empty((k, ldq), dtype=L.code_dtype(pv), device=dev)
    Us = torch.empty((m,), dtype=torch.float32, device=dev)
    Vs = torch.empty((k,), dtype=torch.float32, device=dev)
    Xr = torch.empty((m, k), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    nul = None

    def call(pl, X, recon):
        L._check(lib.lramm_qsvd(pl.handle, 0, L._ptr(X), pu, pv, L._ptr(Uc), L._ptr(Us), L._ptr(Vc), L._ptr(Vs),
                                ldq, L._ptr(nul), L._ptr(nul), L._ptr(Xr if recon else None), k, L._ptr(ws),
                                ws.numel(), L._stream()), "lramm_qsvd")

    for _ in range(max(args.warmup, 0)):
        call(plan, A, False)
    info = L.info_read(ws, 3)
    st = L.status_read(ws)
    if st != 0:
        raise RuntimeError("device status %d after warm-up" % st)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    gpu_id = local
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    n_launch0 = L.launch_count()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        call(plan, A, False)
        ends[i].record(stream)
    n_launch = L.launch_count() - n_launch0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in zip(starts, ends)), dist, dev)
    ms_step = total_ms / args.steps
    value = world * m * k * args.steps / (total_ms * 1e-3) / 1e9
    st = L.status_read(ws)

    # per-kind breakdown with the approximation (instrumented plan, outside the timed region)
    kinds = {}
    nbd = min(args.steps, 5)
    for _ in range(nbd):
        flush.zero_()
        call(tplan, A, True)
        for kname, (ms, cnt) in tplan.timing().items():
            a = kinds.setdefault(kname, [0.0, 0])
            a[0] += ms
            a[1] += cnt

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    t_recon = timed(lambda: call(plan, A, True))
    err = ((Xr.double() - A.double()).norm() / A.double().norm()).item()
    sig = workloads.spectrum(cfg["spectrum"], min(m, k))
    tail = float(np.sqrt(np.sum(sig[r:] ** 2) / np.sum(sig ** 2)))
    # the approximation's product alone: HBM-bound (m k FP32 written, codes read)
    rk = kinds.get("reconstruct")
    pk, peak_src = peaks()
    recon_roof = None
    if rk:
        # the product kernel is the last "reconstruct" launch; its time is the kind's
        # time less the code conversion (a copy of k x ldq codes, timed together)
        rb = m * k * 4 + (m + k) * ldq * 2
        rs = rk[0] / nbd * 1e-3
        recon_roof = {"bound": "hbm", "achieved": rb / rs / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                      "frac": rb / rs / 1e9 / pk["hbm_gbs"], "avg_ms_per_step": rs * 1e3,
                      "algorithmic_bytes": rb, "launches_per_step": rk[1] / nbd,
                      "note": "conversion + product launches of one call together"}
    dname, (dms, dcnt) = max(kinds.items(), key=lambda kv: kv[1][0])
    avg_s = dms / dcnt * 1e-3
    if dname == "svd":
        jf = jacobi_work(l, [int(x) for x in info[1:2] if int(x) > 0])
        roof = {"bound": "alu", "achieved": jf / avg_s / 1e12,
                "peak": fp32_alu_peak_tflops(pk.get("sm_max_mhz", 2070.0)), "unit": "TFLOP/s",
                "kernel": dname, "launches_per_step": dcnt / nbd, "avg_launch_ms": avg_s * 1e3,
                "peak_source": "derived: 152 SM x 128 FP32 FMA x 2 x sm_max_mhz",
                "traffic": measured_traffic("lramm_4096", "svd"), "algorithmic_flops_per_launch": jf}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        roof = {"bound": None, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
                "kernel": dname, "launches_per_step": dcnt / nbd, "avg_launch_ms": avg_s * 1e3}

    # end to end: the matrix in from pinned host memory, codes and scales out
    Ah = A.cpu().pin_memory()
    Ad = torch.empty_like(A)
    outs = [(Uc, torch.empty(Uc.shape, dtype=Uc.dtype).pin_memory()),
            (Vc, torch.empty(Vc.shape, dtype=Vc.dtype).pin_memory()),
            (Us, torch.empty(Us.shape, dtype=Us.dtype).pin_memory()),
            (Vs, torch.empty(Vs.shape, dtype=Vs.dtype).pin_memory())]

    def e2e_step():
        Ad.copy_(Ah, non_blocking=True)
        call(plan, Ad, False)
        for d_, h_ in outs:
            h_.copy_(d_, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e2e_steps = max(2, min(args.steps, 5))
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    eb.record(stream)
    eb.synchronize()
    e2e_ms = ea.elapsed_time(eb) / e2e_steps

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on the full 4096 x 4096 matrix: one step is a few seconds of host work
        Ac, cs = qsvd_cpu_sample(full=True)
        ts_cpu = []
        while sum(ts_cpu) < 10.0 and len(ts_cpu) < 20:    # about 10 s of host work
            ts_cpu.append(cpu_qsvd_step(Ac, cs, (pu, pv)))
        t_cpu = sum(ts_cpu) / len(ts_cpu)
        cpu = {"value": cs["m"] * cs["k"] / t_cpu / 1e9, "unit": "Gentries/s", "cores": cores_used(),
               "kind": "oracle", "sample": "%d oracle Algorithm 4 steps on the full %d x %d matrix, r=%d p=%d q=%d, "
                                             "%.2f s each" % (len(ts_cpu), cs["m"], cs["k"], cs["r"], cs["p"],
                                                              cs["q"], t_cpu)}
    if rank == 0:
        bits = {1: "int8", 2: "int4", 3: "e4m3"}
        line = {
            "metric": QSVD_METRIC, "value": value, "unit": "Gentries/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+%s+%s" % (bits[pu], bits[pv]), "data": "synthetic",
            "config": {"workload": "qsvd_4096", "m": m, "n": k, "r": r, "p": p, "q": q,
                       "d1": bits[pu], "d2": bits[pv], "scale": "per row", "spectrum": cfg["spectrum"],
                       "sketch": sketch_name,
                       "l2": "flushed: 256 MB write before each step", "jacobi_sweeps": info[1:2],
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "with_reconstruction_ms": t_recon,
                       "rel_fro_err_vs_input": err, "rank_r_truncation_floor": tail,
                       "compressed_bytes": Uc.numel() * Uc.element_size() + Vc.numel() * Vc.element_size()
                       + 4 * (m + k), "device_status": st},
            "breakdown_ms_per_step": {kn: round(v[0] / nbd, 4) for kn, v in
                                      sorted(kinds.items(), key=lambda kv: -kv[1][0])},
            "breakdown_note": "CUDA events around every kernel of %d separate steps with the approximation" % nbd,
            "roofline": roof,
            "kernel_rooflines": {"reconstruct": recon_roof} if recon_roof else {},
            "cpu_baseline": cpu,
            "e2e": {"value": world * m * k / (e2e_ms * 1e-3) / 1e9, "unit": "Gentries/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": A.numel() * A.element_size(),
                    "d2h_bytes_per_step": sum(d_.numel() * d_.element_size() for d_, _ in outs)},
            "gpu_launches": n_launch,
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons"), "samples": clk.get("samples")},
            "peaks": peak_src,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["lramm", "reference"], default="lramm")
    ap.add_argument("--workload", default="lramm_32768", choices=sorted(workloads.CONFIGS))
    ap.add_argument("--variant", default="int8", choices=sorted(VARIANTS))
    ap.add_argument("--sketch", choices=["tf32", "fp32", "e4m3"], default=None,
                    help="products with A and B: tf32 tensor cores (default for quantised variants), fp32, or "
                         "e4m3 (the range-finder passes on FP8 codes, the projection in tf32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mn-div", type=int, default=1,
                    help="run a reduced instance of an lramm_* workload: m and n divided by this (k, r, p, q "
                         "kept); the JSON line then names the reduced sizes (profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "rf_linear":
        return run_rf(args)
    if args.workload == "qsvd_4096":
        return run_qsvd(args)
    return run_lramm(args)


if __name__ == "__main__":
    sys.exit(main())
