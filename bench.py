#!/usr/bin/env python
"""Benchmark of the randomized (ST-)HOSVD path on GB300.

Headline workload (one "step" = one batch covering every step of the path):
randomized ST-HOSVD (Algorithm 2, and Algorithm 5 with AMM) of 1024 x 1024 x 512
FP32 video-like tensors (a sum of 50 separable sinusoids plus N(0, 1e-2) noise,
2.15 GB each), ranks (64, 64, 32), P = 16, q = 1, variants
  1. q = 1, no sampling                        (Algorithm 2)
  2. q = 1, c = 20000 fibers, uniform p        (Algorithm 5)
sixteen decompositions of each variant per step, each on its own tensor (32
distinct 2.15 GB tensors, larger than the 129 MB L2, so no flush is needed; one
stream per decomposition, as many as CUDA's hardware work queues), in every
sketch arithmetic (single-pass BF16, TF32, split BF16, FP32). Each
decomposition's orthonormalisations are serial work on a few SMs, so the batch
runs near the streaming bound only when many decompositions share a step
(measured, single-pass BF16: 8 per step 694/s, 16 802/s, 32 834/s).
value = decompositions per second with the tensors resident in HBM, for the
fastest arithmetic whose relative error (Eq. 8) is within 1e-3 of the FP64
oracle's on every variant; the oracle runs on the host on the same bytes (the
first tensor), which also gives the CPU baseline. e2e = the same through the
library's request loop with pinned host buffers (host->device copy of each
input and device->host copy of the factors and core inside the timed region;
four requests of each variant per step), beside the host link's measured rate,
the rate it bounds and the same steps' copies alone.

Secondary lines, each with its own oracle check: the 400^3 batch (low-rank
and Hilbert tensors, q = 1 / 2, AMM c = 4000; 32 distinct buffers), the same
low-rank tensors in the related form (Algorithm 7), fixed-precision ranks
(Problem 2) on a 256^3 tensor beside the oracle's ranks, the 96^4
decaying-core tensor (q = 2), the FP64 100^3 T-HOSVD, randomized T-HOSVD;
the latency of one decomposition alone (headline tensor and 400^3, headline
arithmetic and FP32); and the serving stream (2000 requests of orders 3 and 4, extents up to 256,
a 40 GB admission budget): saturation throughput and p50/p99 latency under
Poisson arrivals, in the headline arithmetic and in FP32.

--impl reference times the FP64 CPU oracle on the headline workload (one
decomposition per step, cycling through the variants).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# A batch runs its decompositions on up to 32 streams of one CUDA graph. CUDA
# maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware work queues (8 unless
# set), and work of different streams sharing a queue is dispatched in order,
# so with 8 a decomposition waiting on its own chain holds up others queued
# behind it. 32 queues give every stream its own; the variable is read when the
# CUDA context is created, so it is set before anything touches the GPU.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

SEED = 0
BASELINE_METRIC = "decomps/s & sketch HBM GB/s, BF16 vs FP32 at equal rel err; serving p50/p99 ms"
FORMS = ["bf16x1", "tf32", "bf16", "fp32"]
RE_GATE = 1e-3            # reduced-precision forms: |RE - RE_oracle|
FP32_RE_BAR = 1e-5        # exact FP32 form, where the sketch is not rank-deficient

WORKLOADS = {
    "video1024": dict(
        desc="randomized ST-HOSVD of 1024x1024x512 FP32 video-like tensors (sum of 50 separable sinusoids + "
             "N(0,1e-2) noise, 2.15 GB each), R=(64,64,32) P=16 q=1; variants: Algorithm 2; Algorithm 5 with "
             "c=20000 uniform",
        which="ST", dims=(1024, 1024, 512), ranks=(64, 64, 32), P=16, dtype="f32", copies=16,
        variants=[dict(name="q1", gen="video", q=1, c=0, prob="uniform"),
                  dict(name="q1_amm20000_uniform", gen="video", q=1, c=20000, prob="uniform")]),
    "cube400": dict(
        desc="randomized ST-HOSVD of 400^3 FP32 tensors (Tucker core 20^3 + 1e-2 noise, and the Hilbert tensor "
             "1/(i+j+k-2)), R=20 P=10; variants: q=1; q=1 AMM c=4000 nearly-optimal; Hilbert q=2; Hilbert q=1 "
             "AMM c=4000 uniform",
        which="ST", dims=(400, 400, 400), ranks=(20, 20, 20), P=10, dtype="f32", copies=8,
        variants=[dict(name="lowrank_q1", gen="lowrank", q=1, c=0, prob="uniform"),
                  dict(name="lowrank_q1_amm4000_nearly_optimal", gen="lowrank", q=1, c=4000, prob="nearly_optimal"),
                  dict(name="hilbert_q2", gen="hilbert", q=2, c=0, prob="uniform", rank_deficient=True),
                  dict(name="hilbert_q1_amm4000_uniform", gen="hilbert", q=1, c=4000, prob="uniform",
                       rank_deficient=True)]),
    # Algorithms 6/7 (the related forms): P_n from the paper-form sketch by CholeskyQR2, one more power
    # step, the leading vectors of the L x L matrix P^T A A^T P, Q_n = P U
    "cube400_related": dict(
        desc="randomized ST-HOSVD of 400^3 FP32 low-rank tensors (Tucker core 20^3 + 1e-2 noise) in the related "
             "form (Algorithm 7), R=20 P=10 q=1",
        which="ST", dims=(400, 400, 400), ranks=(20, 20, 20), P=10, dtype="f32", copies=16, form="related",
        forms=["bf16x1", "fp32"],
        variants=[dict(name="lowrank_q1_related", gen="lowrank", q=1, c=0, prob="uniform")]),
    "quartic96": dict(
        desc="randomized ST-HOSVD of 96^4 FP32 tensors with a decaying 16^4 core (entries N(0,1) 0.8^(i1+i2+i3+i4), "
             "no noise), R=16 P=8 q=2",
        which="ST", dims=(96, 96, 96, 96), ranks=(16, 16, 16, 16), P=8, dtype="f32", copies=16,
        variants=[dict(name="q2", gen="decaying", q=2, c=0, prob="uniform")]),
    "fp64cube100": dict(
        desc="randomized T-HOSVD of 100^3 FP64 tensors (Tucker core 10^3 + 1e-3 noise), R=10 P=5 q=1",
        which="T", dims=(100, 100, 100), ranks=(10, 10, 10), P=5, dtype="f64", copies=32, forms=["fp32"],
        flush_l2=True,
        variants=[dict(name="q1", gen="lowrank64", q=1, c=0, prob="uniform")]),
    # the headline tensors in the range form: Y = A_(n) Omega with Omega (J_n x L) generated per tile inside
    # the tensor-core kernel, then one power step A_(n)(A_(n)^T orth(Y))
    "video1024_range": dict(
        desc="randomized ST-HOSVD of 1024x1024x512 FP32 video-like tensors in the range form (Y = A_(n) Omega, "
             "Omega J_n x L generated in-kernel, then q=1 power step), R=(64,64,32) P=16",
        which="ST", dims=(1024, 1024, 512), ranks=(64, 64, 32), P=16, dtype="f32", copies=4, form="range",
        forms=["bf16x1", "fp32"],
        variants=[dict(name="range_q1", gen="video", q=1, c=0, prob="uniform")]),
    # a smaller tensor with the headline's mode-1 shapes (I_1 = 1024, L_1 = 80, R_1 = 64; 268 MB, still
    # larger than L2): the case for profiler captures of the headline's kernels (--single only)
    "video1024x256": dict(
        desc="randomized ST-HOSVD of a 1024x256x256 FP32 video-like tensor, R=(64,64,32) P=16 q=1 (profiling case)",
        which="ST", dims=(1024, 256, 256), ranks=(64, 64, 32), P=16, dtype="f32", copies=1, profile_only=True,
        variants=[dict(name="q1", gen="video", q=1, c=0, prob="uniform"),
                  dict(name="q1_amm20000_uniform", gen="video", q=1, c=20000, prob="uniform")]),
}
HEADLINE = "video1024"


# ---------------------------------------------------------------- inputs
def reference_tensor(gen, dims):
    """The first tensor of a generator (seed 0), built on the host with numpy:
    the bytes both the GPU path and the oracle decompose."""
    import numpy as np
    import synth
    if gen == "video":
        return synth.flat(synth.video_like(dims, seed=SEED))
    if gen == "lowrank":
        return synth.flat(synth.lowrank_noise(dims, (20,) * len(dims), rel_noise=1e-2, seed=SEED))
    if gen == "hilbert":
        return synth.flat(synth.hilbert(dims))
    if gen == "decaying":
        return synth.flat(synth.decaying_core(dims, 16, ratio=0.8, seed=SEED))
    if gen == "lowrank64":
        return synth.flat(synth.lowrank_noise(dims, (10,) * len(dims), rel_noise=1e-3, seed=SEED, dtype=np.float64))
    raise ValueError(gen)


def slot_tensor(torch, gen, dims, k, ref_dev):
    """Tensor k >= 1 of a generator, built on the device with the same recipe
    (distinct values; the Hilbert tensor is deterministic, so its slots hold
    copies in distinct buffers)."""
    import numpy as np
    import synth
    from synth import device as sd
    if gen == "video":
        return sd.video_like(torch, dims, seed=SEED + k)
    if gen == "lowrank":
        return sd.tucker_tensor(torch, dims, (20,) * len(dims), 1e-2, seed=SEED + k)
    if gen == "hilbert":
        return ref_dev.clone()
    if gen == "decaying":
        idx = np.meshgrid(*[np.arange(16)] * len(dims), indexing="ij")
        return sd.tucker_tensor(torch, dims, (16,) * len(dims), 0.0, seed=SEED + k, core_scale=0.8 ** sum(idx))
    if gen == "lowrank64":
        return torch.from_numpy(synth.flat(synth.lowrank_noise(dims, (10,) * len(dims), rel_noise=1e-3,
                                                               seed=SEED + k, dtype=np.float64))).cuda()
    raise ValueError(gen)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.active = False

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            if self.active:
                self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "samples taken while timed regions ran"}


# ---------------------------------------------------------------- oracle (CPU baseline and accuracy reference)
def oracle_run(W, v, host_ref):
    """One oracle decomposition of variant v on the reference tensor: (Us, G, RE, seconds)."""
    import numpy as np
    import synth
    from oracle import tucker as ot
    A = synth.from_flat(host_ref, W["dims"]).astype(np.float64)
    t0 = time.perf_counter()
    fn = ot.rsthosvd if W["which"] == "ST" else ot.rthosvd
    Us, G = fn(A, W["ranks"], P=W["P"], q=v["q"], c=v["c"], prob=v["prob"], seed=SEED, form=W.get("form", "paper"))
    dt = time.perf_counter() - t0
    re = ot.relative_error(A, Us, G) if A.size <= 100_000_000 else \
        math.sqrt(max(0.0, 1.0 - ot.frobenius(G) ** 2 / ot.frobenius(A) ** 2))
    return Us, np.asarray(G).reshape(-1, order="F"), re, dt


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_one_thread(workload, variant, timeout_s=120):
    """The oracle on one host thread (the paper's setting, maxNumCompThreads = 1),
    one decomposition of a variant, timed in a fresh process whose BLAS is held
    to one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    code = ("import sys, json; sys.path.insert(0, sys.argv[1]); import bench; "
            "W = bench.WORKLOADS[sys.argv[2]]; v = next(x for x in W['variants'] if x['name'] == sys.argv[3]); "
            "ref = bench.reference_tensor(v['gen'], W['dims']); _, _, re, dt = bench.oracle_run(W, v, ref); "
            "print(json.dumps({'seconds': dt, 're': re}))")
    try:
        out = subprocess.run([sys.executable, "-c", code, ROOT, workload, variant], env=env, capture_output=True,
                             text=True, timeout=timeout_s)
        r = json.loads(out.stdout.strip().splitlines()[-1])
        return {"value": 1.0 / r["seconds"], "unit": "decomps/s", "cores": 1, "kind": "oracle",
                "sample": f"one {workload} {variant} decomposition on one thread ({r['seconds']:.1f} s)"}
    except Exception as exc:  # noqa: BLE001
        return {"value": None, "unit": "decomps/s", "cores": 1, "kind": "oracle", "error": str(exc)[:200]}


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank):
    if rank != 0:
        return 0
    W = WORKLOADS[HEADLINE]
    refs = {}
    for v in W["variants"]:
        if v["gen"] not in refs:
            refs[v["gen"]] = reference_tensor(v["gen"], W["dims"])
    vs = W["variants"]
    for k in range(args.warmup):
        oracle_run(W, vs[k % len(vs)], refs[vs[k % len(vs)]["gen"]])
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle_run(W, vs[k % len(vs)], refs[vs[k % len(vs)]["gen"]])
    dt = time.perf_counter() - t0
    val = args.steps / dt
    line = {"impl": "reference", "metric": "decomps/s", "value": val, "unit": "decomps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "baseline_metric": BASELINE_METRIC,
            "config": {"workload": W["desc"] + " (reference: FP64 CPU oracle, one decomposition per step)"},
            "cpu_baseline": {"value": val, "unit": "decomps/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{args.steps} decompositions cycling through the {len(vs)} variants"},
            "e2e": {"value": val, "unit": "decomps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- serving
SERVE_N = 2000
SERVE_BUDGET = 40 << 30
SERVE_RESIDENT = 48 << 30


def serving_specs(n=SERVE_N, seed=0):
    """The serving stream of the config: n randomized ST-HOSVD requests (P = 5, q = 1), order 3 or 4 with
    equal odds, every extent uniform in 32..256, ranks uniform in 4..32 (at most the extent), each a
    low-rank (core of the ranks) plus 1e-2 noise FP32 tensor; order-4 requests reach 256^4 = 17 GB."""
    import synth
    return synth.serving_requests(n, seed=seed, dim_range=(32, 256), rank_range=(4, 32), orders=(3, 4))


def serving_batches(specs, resident=SERVE_RESIDENT):
    """Consecutive groups of the stream whose inputs fit `resident` bytes of device memory together."""
    import numpy as np
    out, cur, used = [], [], 0
    for r in specs:
        b = 4 * int(np.prod(r["dims"]))
        if cur and used + b > resident:
            out.append(cur)
            cur, used = [], 0
        cur.append(r)
        used += b
    if cur:
        out.append(cur)
    return out


def serving_inputs(torch, batch):
    """The batch's tensors, generated on the device (untimed; they stand for data that has arrived in HBM)."""
    from synth import device as sd
    xs = [sd.tucker_tensor_lean(torch, r["dims"], r["ranks"], 1e-2, seed=1000 + r["id"]) for r in batch]
    torch.cuda.synchronize()
    return xs


def serving_bench(tk, torch, specs, prec, load=0.7):
    """The whole stream through one server per phase, in groups of requests whose inputs are generated on
    the device before the group (outside the timed region). Saturation: each group submitted at once, the
    rate over the groups' wall times. Latency: within each group arrivals are Poisson at `load` times the
    saturation rate (the queue drains between groups); p50/p99 over every request, submission to
    completion, as the server records them."""
    import numpy as np
    batches = serving_batches(specs)
    sat_s, n = 0.0, 0
    with tk.Server(budget_bytes=SERVE_BUDGET, max_inflight=16, prec=prec) as srv:
        for batch in batches:
            xs = serving_inputs(torch, batch)
            t0 = time.perf_counter()
            ts = [srv.submit("ST", x, r["dims"], r["ranks"], P=5, q=1, seed=r["seed"]) for x, r in zip(xs, batch)]
            for t in ts:
                srv.wait(t)
            sat_s += time.perf_counter() - t0
            n += len(batch)
            del xs, ts
        sat_peak = srv.stats()["peak_bytes"]
    sat = n / sat_s
    rate = load * sat
    rng = np.random.default_rng(1)
    busy_s = 0.0
    with tk.Server(budget_bytes=SERVE_BUDGET, max_inflight=16, prec=prec) as srv:
        for batch in batches:
            xs = serving_inputs(torch, batch)
            gaps = rng.exponential(1.0 / rate, size=len(batch))
            t0 = time.perf_counter()
            due = t0
            ts = []
            for x, r, gap in zip(xs, batch, gaps):
                due += gap
                while time.perf_counter() < due:
                    pass
                ts.append(srv.submit("ST", x, r["dims"], r["ranks"], P=5, q=1, seed=r["seed"]))
            for t in ts:
                srv.wait(t)
            busy_s += time.perf_counter() - t0
            del xs, ts
        st = srv.stats()
    return {"requests": n, "groups": len(batches), "saturation_decomps_per_s": sat, "offered_per_s": rate,
            "decomps_per_s": n / busy_s, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "max_ms": st["max_ms"], "peak_inflight": st["peak_inflight"],
            "peak_bytes": max(st["peak_bytes"], sat_peak), "failed": st["failed"]}


# ---------------------------------------------------------------- latency
def latency_bench(tk, torch, stream, precs):
    """One decomposition alone, as a caller waiting for its result sees it: randomized ST-HOSVD (q = 1) of the
    headline's 1024 x 1024 x 512 video-like tensor (R = (64, 64, 32), P = 16) and of a 400^3 low-rank tensor
    (R = 20, P = 10), input resident in HBM, asynchronous call into a preallocated workspace on one stream,
    CUDA events around it; 2 warm-up calls, then the median and minimum of 5."""
    import numpy as np
    import synth
    from synth import device as sd
    cases = {"video1024": ((1024, 1024, 512), (64, 64, 32), 16,
                           lambda: sd.video_like(torch, (1024, 1024, 512), seed=SEED)),
             "cube400": ((400, 400, 400), (20, 20, 20), 10,
                         lambda: torch.from_numpy(synth.flat(synth.lowrank_noise((400,) * 3, (20,) * 3, rel_noise=1e-2,
                                                                                  seed=SEED))).cuda())}
    out = {}
    for name, (dims, ranks, P, make) in cases.items():
        A = make()
        # outputs allocated once; everything generated on the default stream is complete
        # before the decompositions on `stream` read it
        U = [torch.empty((R, I), dtype=torch.float32, device="cuda").t() for I, R in zip(dims, ranks)]
        G = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        res = {"workload": f"randomized ST-HOSVD of {'x'.join(map(str, dims))}, R={ranks}, P={P}, q=1"}
        for prec in precs:
            ws = torch.empty(tk.workspace_size("ST", dims, ranks, P=P, q=1, prec=prec), dtype=torch.uint8,
                             device="cuda")
            torch.cuda.synchronize()
            ms = []
            for k in range(7):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                tk.decompose("ST", A, dims, ranks, P=P, q=1, seed=SEED, prec=prec, stream=stream, workspace=ws,
                             flags=tk.FLAG_ASYNC, out=(U, G))
                e1.record(stream)
                stream.synchronize()
                if k >= 2:
                    ms.append(e0.elapsed_time(e1))
            # the last call's status (0: ok; 4: TUCKER_ERR_NUMERICAL, a sketch CholeskyQR could not
            # orthonormalise even shifted; 5: a bounded wait ran out)
            res[prec] = {"median_ms": float(np.median(ms)), "min_ms": float(min(ms)),
                         "status": int(tk.last_device_status())}
            del ws
        out[name] = res
        del A
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- fusions
def fusion_bench(tk, torch, stream):
    """The fiber norms of a 400^3 FP32 tensor (Algorithm 4's nearly-optimal probabilities): modes 1 and 2
    in one fused pass against two per-mode passes, and all three modes in one pass (plus the sums of its
    partials) against three; kernel time from the library's per-launch CUDA events (profile class
    "norms"), 2 warm-up calls, then 7 of each."""
    import synth
    dims = (400, 400, 400)
    A = torch.from_numpy(synth.flat(synth.lowrank_noise(dims, (20,) * 3, rel_noise=1e-2, seed=SEED))).cuda()
    torch.cuda.synchronize()

    def timed(fn, launches):
        for _ in range(2):
            fn()
        tk.profile_enable(True)
        for _ in range(7):
            fn()
        n, ms, _, _ = tk.profile_read("norms")
        tk.profile_enable(False)
        if n != 7 * launches:
            raise RuntimeError(f"expected {7 * launches} norm launches, profiled {n}")
        return ms / 7

    fused = timed(lambda: tk.fiber_norms12(A, dims, stream=stream), 1)
    apart = timed(lambda: (tk.fiber_norms(A, dims, 0, stream=stream), tk.fiber_norms(A, dims, 1, stream=stream)), 2)
    ws = torch.empty(tk.fiber_norms123_workspace_size(dims), dtype=torch.uint8, device="cuda")
    all3 = timed(lambda: tk.fiber_norms123(A, dims, stream=stream, workspace=ws), 1)
    apart3 = timed(lambda: [tk.fiber_norms(A, dims, n, stream=stream) for n in range(3)], 3)
    gb = A.numel() * 4 / 1e9
    return {"norms12_400cubed": {"workload": "squared fiber norms of modes 1 and 2 of a 400^3 FP32 tensor",
                                 "fused_ms": fused, "per_mode_ms": apart, "fused_gbs": gb / (fused * 1e-3),
                                 "speedup": apart / fused},
            "norms123_400cubed": {"workload": "squared fiber norms of all three modes of a 400^3 FP32 tensor "
                                              "(one pass over the tensor, then the partials summed)",
                                  "fused_ms": all3, "per_mode_ms": apart3, "fused_gbs": gb / (all3 * 1e-3),
                                  "speedup": apart3 / all3}}


def adaptive_bench(tk, torch, precs):
    """Fixed-precision ranks (Problem 2, tucker_rsthosvd_adaptive) on a 256^3 FP32 low-rank tensor (Tucker
    core 16^3 + 1e-2 noise) at eps = 2e-2: ranks and relative error beside the oracle's on the same bytes,
    and the call's wall time (it decides each mode's rank on the host between modes), 2 warm-up calls,
    then the median of 7."""
    import numpy as np
    import synth
    from oracle import tucker as ot
    dims, eps = (256, 256, 256), 2e-2
    host = synth.flat(synth.lowrank_noise(dims, (16, 16, 16), rel_noise=1e-2, seed=SEED))
    A = torch.from_numpy(host).cuda()
    A64 = synth.from_flat(host, dims).astype(np.float64)
    t0 = time.perf_counter()
    Qo, Go, ro = ot.rsthosvd_adaptive(A64, eps, q=1, seed=SEED)
    t_or = time.perf_counter() - t0
    out = {"workload": f"fixed-precision ST-HOSVD (Problem 2) of a 256^3 FP32 low-rank tensor, eps={eps}, q=1, "
                       f"L0=8", "oracle_ranks": [int(r) for r in ro],
           "oracle_rel_error": ot.relative_error(A64, Qo, Go), "oracle_seconds": t_or}
    for prec in precs:
        ts, res = [], None
        for it in range(9):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            res = tk.rsthosvd_adaptive(A, dims, eps, q=1, seed=SEED, prec=prec, want_rel_error=True)
            ts.append(time.perf_counter() - t1)
        U, G, ranks, re = res
        ms = 1e3 * sorted(ts[2:])[len(ts[2:]) // 2]
        out[prec] = {"ms_per_call": ms, "decomps_per_s": 1e3 / ms, "ranks": [int(r) for r in ranks],
                     "rel_error": re, "ranks_equal_oracle": [int(r) for r in ranks] == [int(r) for r in ro]}
    return out


# ---------------------------------------------------------------- ranks
def rank_barrier(dist, torch, cuda=True):
    """Every rank's queued GPU work done, then all ranks meet (timed regions
    start and end here)."""
    if cuda:
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    if cuda:
        torch.cuda.synchronize()


def rank_max(dist, torch, x, device):
    """Largest value over the ranks (the slowest rank's time)."""
    if not dist:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Weak scaling: every rank processes units_per_rank; the job takes the
    slowest rank's time."""
    return units_per_rank * world / seconds


# ---------------------------------------------------------------- accuracy against the oracle
def projector_distance(U, Uo):
    """||U U^T - Uo Uo^T||_2 for orthonormal I x R bases: the sine of the largest
    principal angle, sqrt(1 - sigma_min(U^T Uo)^2)."""
    import numpy as np
    s = np.linalg.svd(U.T @ Uo, compute_uv=False)
    return float(math.sqrt(max(0.0, 1.0 - float(np.min(s)) ** 2)))


# ---------------------------------------------------------------- GPU arm
class Bench:
    def __init__(self, args, torch, tk, dist, world):
        self.args, self.torch, self.tk, self.dist, self.world = args, torch, tk, dist, world
        self.main_s = torch.cuda.Stream()
        self.clocks = None

    def barrier(self):
        rank_barrier(self.dist, self.torch, cuda=True)

    def max_over_ranks(self, x):
        return rank_max(self.dist, self.torch, x, "cuda")

    def prepare(self, name):
        """Reference tensors (host, seed 0) with their oracle results, and one
        distinct device tensor per batch slot."""
        import numpy as np
        torch = self.torch
        W = WORKLOADS[name]
        refs, oracle = {}, {}
        t_oracle = 0.0
        for v in W["variants"]:
            if v["gen"] not in refs:
                refs[v["gen"]] = reference_tensor(v["gen"], W["dims"])
            Us, G, re, dt = oracle_run(W, v, refs[v["gen"]])
            oracle[v["name"]] = dict(U=Us, G=G, re=re, seconds=dt)
            t_oracle += dt
        ref_dev = {g: torch.from_numpy(h).cuda() for g, h in refs.items()}
        slots, counts = [], {}
        for v in W["variants"]:
            for _ in range(W["copies"]):
                k = counts.get(v["gen"], 0)
                counts[v["gen"]] = k + 1
                A = ref_dev[v["gen"]] if k == 0 else slot_tensor(torch, v["gen"], W["dims"], k, ref_dev[v["gen"]])
                slots.append((v, A))
        torch.cuda.synchronize()
        return dict(W=W, refs=refs, ref_dev=ref_dev, oracle=oracle, slots=slots, oracle_seconds=t_oracle,
                    distinct=sum(counts.values()))

    def accuracy(self, P, prec):
        """RE (explicit reconstruction on the device) of every variant on the
        reference tensor, with its distance to the oracle's, projector distances
        per mode and the core's relative error."""
        import numpy as np
        tk, W = self.tk, P["W"]
        out = {}
        for v in W["variants"]:
            A = P["ref_dev"][v["gen"]]
            U, G = tk.decompose(W["which"], A, W["dims"], W["ranks"], P=W["P"], q=v["q"], c=v["c"], prob=v["prob"],
                                form=W.get("form", "paper"),
                                seed=SEED, prec=prec)
            re = tk.relative_error(A, W["dims"], W["ranks"], U, G)
            o = P["oracle"][v["name"]]
            Uh = [u.double().cpu().numpy() for u in U]
            Gh = G.double().cpu().numpy()
            out[v["name"]] = {
                "rel_error": re, "oracle_rel_error": o["re"], "abs_diff": abs(re - o["re"]),
                "projector_dist": [projector_distance(u, uo) for u, uo in zip(Uh, o["U"])],
                "core_rel_err": float(np.linalg.norm(Gh - o["G"]) / max(np.linalg.norm(o["G"]), 1e-300))}
        return out

    def timed(self, P, prec, steps):
        """Graph-timed throughput of the batch (every slot its own tensor)."""
        torch, tk, W = self.torch, self.tk, P["W"]
        bt = tk.Batch([dict(which=W["which"], A=A, dims=W["dims"], ranks=W["ranks"], P=W["P"], q=v["q"], c=v["c"],
                            prob=v["prob"], seed=SEED) for v, A in P["slots"]], prec=prec,
                      form=W.get("form", "paper"))
        for _ in range(self.args.warmup):
            bt.run(stream=self.main_s, sync=False)
        self.main_s.synchronize()
        bt.run(stream=self.main_s)                               # synchronous: raises on a device status
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda") if W.get("flush_l2") else None
        self.barrier()
        self.clocks.active = True
        n0 = tk.launch_count()
        ms = 0.0
        if flush is None:
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(self.main_s)
            for _ in range(steps):
                bt.run(stream=self.main_s, sync=False)
            ev1.record(self.main_s)
            self.main_s.synchronize()
            ms = ev0.elapsed_time(ev1)
        else:
            # small tensors: the L2 is flushed between steps, outside the timed events
            evs = []
            with torch.cuda.stream(self.main_s):
                for _ in range(steps):
                    flush.fill_(1)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(self.main_s)
                    bt.run(stream=self.main_s, sync=False)
                    e1.record(self.main_s)
                    evs.append((e0, e1))
            self.main_s.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs)
        n1 = tk.launch_count()
        self.clocks.active = False
        self.barrier()
        if any(bt.status()):
            raise RuntimeError("device status not OK in the timed region")
        ms = self.max_over_ranks(ms)
        del bt
        return {"ms": ms, "value": whole_job_rate(len(P["slots"]) * steps, self.world, ms / 1e3),
                "gpu_launches": n1 - n0}

    def profile(self, P, prec, reps):
        """Per-kernel-class launch counts, times and algorithmic bytes/flops from
        eager decompositions run one at a time on one stream (graph-captured
        event pairs carry no timings)."""
        import numpy as np
        torch, tk, W = self.torch, self.tk, P["W"]
        wss, outs = [], []
        for v in W["variants"]:
            dt = P["ref_dev"][v["gen"]].dtype
            wss.append(torch.empty(tk.workspace_size(W["which"], W["dims"], W["ranks"], P=W["P"], q=v["q"], c=v["c"],
                                                     dtype=dt, prec=prec, form=W.get("form", "paper")),
                                   dtype=torch.uint8, device="cuda"))
            outs.append(([tk.factor_tensor(I, R, dt, "cuda") for I, R in zip(W["dims"], W["ranks"])],
                         torch.empty(int(np.prod(W["ranks"])), dtype=dt, device="cuda")))
        tk.profile_enable(True)
        for _ in range(reps):
            for v, ws, out in zip(W["variants"], wss, outs):
                tk.decompose(W["which"], P["ref_dev"][v["gen"]], W["dims"], W["ranks"], P=W["P"], q=v["q"], c=v["c"],
                             prob=v["prob"], seed=SEED, workspace=ws, stream=self.main_s, out=out,
                             flags=tk.FLAG_ASYNC, prec=prec, form=W.get("form", "paper"))
        self.main_s.synchronize()
        from paper_2303_11612_gb300 import _binding as B
        prof = {k: tk.profile_read(k) for k in B.KERNEL_CLASSES}
        tk.profile_enable(False)
        if tk.last_device_status() != 0:
            raise RuntimeError("device status not OK in the profiled decompositions")
        return prof

    def full_tensor_profile(self, P, prec, reps=3):
        """Per-class times of the headline's mode-1 launches on the full input tensor alone (one power step
        and one mode product, eager, on one stream): the decomposition profile averages them with the
        small launches on AMM samples and truncated tensors."""
        torch, tk, W = self.torch, self.tk, P["W"]
        from paper_2303_11612_gb300 import _binding as B
        A = P["ref_dev"][W["variants"][0]["gen"]]
        dims = W["dims"]
        L = min(W["ranks"][0] + W["P"], dims[0])
        X = B.gaussian(dims[0], L, SEED, 0, device="cuda", stream=self.main_s)
        U = B.gaussian(dims[0], W["ranks"][0], SEED, 1, device="cuda", stream=self.main_s)
        for _ in range(2):
            B.power_step(A, dims, 0, X, stream=self.main_s, prec=prec)
            B.ttm(A, dims, 0, U, transpose=True, stream=self.main_s, prec=prec)
        self.main_s.synchronize()
        tk.profile_enable(True)
        for _ in range(reps):
            B.power_step(A, dims, 0, X, stream=self.main_s, prec=prec)
            B.ttm(A, dims, 0, U, transpose=True, stream=self.main_s, prec=prec)
        self.main_s.synchronize()
        prof = {k: tk.profile_read(k) for k in B.KERNEL_CLASSES}
        tk.profile_enable(False)
        return prof

    def workload_line(self, name, forms, steps):
        """Every form of one workload: accuracy against the oracle, timed batch,
        and the gates."""
        P = self.prepare(name)
        W = P["W"]
        res = {}
        for prec in forms:
            acc = self.accuracy(P, prec)
            t = self.timed(P, prec, steps)
            gate = all(a["abs_diff"] <= RE_GATE for a in acc.values())
            fp32_bar = {k: a["abs_diff"] <= FP32_RE_BAR for k, a in acc.items()
                        if not next(v for v in W["variants"] if v["name"] == k).get("rank_deficient")}
            res[prec] = dict(t, accuracy=acc, re_within_1e_3_of_oracle=gate,
                             re_within_1e_5_of_oracle=fp32_bar if prec == "fp32" else None)
        return P, res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="all", choices=["all"] + FORMS,
                    help="sketch arithmetic to time (all: the headline is the fastest form whose relative "
                         "errors are within 1e-3 of the oracle's)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-secondary", action="store_true", help="headline workload only")
    ap.add_argument("--copies", type=int, default=0,
                    help="decompositions of each variant per step in the headline batch (0: the workload's "
                         "default), every one on its own tensor")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default kernel configurations (no tuning in the synchronous warm-up calls)")
    ap.add_argument("--single", default=None,
                    help="WORKLOAD:VARIANT[,VARIANT...] -- run one decomposition of each listed variant after one "
                         "warm-up and exit (profiling case)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    args.warmup = max(args.warmup, 3)

    import numpy as np
    import torch
    import paper_2303_11612_gb300 as tk

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.single:
        wname, vnames = args.single.split(":") if ":" in args.single else ("cube400", args.single)
        W = WORKLOADS[wname]
        prec = "bf16x1" if args.prec == "all" else args.prec
        tensors = {}
        for vname in vnames.split(","):
            v = next(x for x in W["variants"] if x["name"] == vname)
            if v["gen"] not in tensors:
                tensors[v["gen"]] = torch.from_numpy(reference_tensor(v["gen"], W["dims"])).cuda()
            # asynchronous calls with a caller workspace: the launch configuration of the timed batch
            ws = torch.empty(tk.workspace_size(W["which"], W["dims"], W["ranks"], P=W["P"], q=v["q"], c=v["c"],
                                               prec=prec), dtype=torch.uint8, device="cuda")
            for _ in range(2):
                tk.decompose(W["which"], tensors[v["gen"]], W["dims"], W["ranks"], P=W["P"], q=v["q"], c=v["c"],
                             prob=v["prob"], seed=SEED, prec=prec, workspace=ws, flags=tk.FLAG_ASYNC)
            torch.cuda.synchronize()
            if tk.last_device_status() != 0:
                raise RuntimeError("device status not OK")
        torch.cuda.synchronize()
        print(json.dumps({"single": args.single, "prec": prec, "ok": True}))
        return 0
    if not args.no_autotune:
        # the synchronous accuracy checks meet every shape class first and tune it;
        # the graph-captured batch steps then reuse the kept choices
        tk.autotune_enable(True)
    b = Bench(args, torch, tk, dist, world)
    b.clocks = ClockSampler(local)
    b.clocks.start()
    forms = FORMS if args.prec == "all" else [args.prec]

    # ---- headline
    if args.copies > 0:
        WORKLOADS[HEADLINE]["copies"] = args.copies
    P, res = b.workload_line(HEADLINE, forms, args.steps)
    W = P["W"]
    ok = {p: r["re_within_1e_3_of_oracle"] for p, r in res.items()}
    cands = [p for p in res if ok[p]] or list(res)
    head = max(cands, key=lambda p: res[p]["value"])
    prof = b.profile(P, head, reps=max(2, args.steps // 10))

    full = b.full_tensor_profile(P, head)

    peaks, peak_kind = load_peaks()
    # the dominant kernel: the streaming class (power steps, mode products) with the largest share of
    # kernel time in the profiled decompositions; the extraction chain is latency-bound (one CTA per
    # step) and overlaps other decompositions' passes in the batch
    stream_classes = [k for k in prof if (k.startswith("power") or k.startswith("ttm") or k == "range_wide")
                      and prof[k][0] > 0]
    pclass = max(stream_classes, key=lambda k: prof[k][1])
    pw_n, pw_ms, pw_bytes, pw_flops = prof[pclass]
    achieved_gbs = pw_bytes / (pw_ms / 1e3) / 1e9 if pw_ms > 0 else 0.0
    achieved_tflops = pw_flops / (pw_ms / 1e3) / 1e12 if pw_ms > 0 else 0.0
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    if pclass not in ("power", "ttm"):
        # bandwidth-bound: 2 L flops per 4-byte element and pass (40 flops/byte at L = 80, 32 for a mode
        # product with K = 64; three products in split bf16) is below the bf16 tensor ridge (~280 flops/byte),
        # so the bound is HBM
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved_gbs / peaks["hbm_gbs"], "kernel_class": pclass, "tensor_tflops": achieved_tflops}
    else:
        fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
        roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": achieved_tflops / fp32_peak, "kernel_class": pclass,
                    "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz", "hbm_gbs": achieved_gbs}
    traffic = None
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f).get(f"{pclass}@{HEADLINE}")
        if tr:
            src = open(os.path.join(ROOT, "paper_2303_11612_gb300", "csrc", tr["source"]), "rb").read()
            if tr.get("source_sha256") == hashlib.sha256(src).hexdigest():
                traffic = tr["dram_bytes_per_algorithmic_byte"] * pw_bytes / max(pw_n, 1)
    except Exception:
        traffic = None
    full_launch = {}
    for k, (n, kms, by, fl) in full.items():
        if n and by:
            gbs = by / (kms / 1e3) / 1e9
            full_launch[k] = {"launches": n, "ms_per_launch": kms / n, "algorithmic_bytes_per_launch": by / n,
                              "achieved_gbs": gbs, "frac": gbs / peaks["hbm_gbs"]}
    roofline["mode1_full_tensor"] = {
        "what": "the headline's mode-1 launches on the full 2.15 GB input alone: one power step (two passes) and "
                "one mode product, eager on one stream, CUDA events around each launch",
        "classes": full_launch}
    roofline.update({"traffic": traffic, "launches": pw_n, "ms_per_launch": pw_ms / max(pw_n, 1),
                     "algorithmic_bytes_per_launch": pw_bytes / max(pw_n, 1), "peak_kind": peak_kind,
                     "timing": "CUDA events on the launching stream around each launch, in eager decompositions "
                               "run one at a time right after the graph-timed region (graph event nodes carry "
                               "no timings)"})
    kernels = {}
    for k, (n, kms, by, fl) in prof.items():
        if n:
            kernels[k] = {"launches": n, "ms_per_launch": kms / n, "share_of_kernel_time":
                          kms / max(sum(x[1] for x in prof.values()), 1e-12)}
            if by:
                kernels[k].update({"gbs": by / (kms / 1e3) / 1e9,
                                   "hbm_frac": by / (kms / 1e3) / 1e9 / peaks["hbm_gbs"]})

    # ---- end to end through the request loop with pinned host buffers, headline arithmetic
    e2e = None
    try:
        # four requests of each variant per step: the host link bounds this path, and more slots
        # would only pin more host memory
        per = min(4, W["copies"])
        e2e_slots = [sl for i, v in enumerate(W["variants"]) for sl in P["slots"][i * W["copies"]:i * W["copies"] + per]]
        host_in = [torch.empty(A.numel(), dtype=A.dtype).pin_memory() for _, A in e2e_slots]
        for h, (_, A) in zip(host_in, e2e_slots):
            h.copy_(A)
        houts = [([torch.empty((R, I), dtype=torch.float32).pin_memory().t() for I, R in zip(W["dims"], W["ranks"])],
                  torch.empty(int(np.prod(W["ranks"])), dtype=torch.float32).pin_memory()) for _ in e2e_slots]
        budget = sum(h.numel() * 4 for h in host_in) + (24 << 30)
        with tk.Server(budget_bytes=budget, max_inflight=len(e2e_slots), prec=head) as srv:
            def step_e2e():
                ts = [srv.submit(W["which"], h, W["dims"], W["ranks"], P=W["P"], q=v["q"], c=v["c"], prob=v["prob"],
                                 seed=SEED, out=out) for (v, _), h, out in zip(e2e_slots, host_in, houts)]
                for t in ts:
                    srv.wait(t)

            # the first passes of the DMA engines over freshly pinned host buffers run at a third of the
            # link's rate (measured: 64, 81, then 211 GB/s over three passes), so the buffers, which a
            # serving process keeps for its lifetime, are warmed by untimed steps; the timed steps are
            # many enough (10 at the default 20) that a step slowed by the shared host moves the rate
            # little (single steps of 124 to 243 ms against 86.5 were seen)
            for _ in range(5):
                step_e2e()
            b.barrier()
            e2e_steps = max(5, args.steps // 2)
            step_ms = []
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                t1 = time.perf_counter()
                step_e2e()
                step_ms.append(round(1e3 * (time.perf_counter() - t1), 1))
            e2e_s = b.max_over_ranks(time.perf_counter() - t0)
        h2d = sum(h.numel() * h.element_size() for h in host_in)
        d2h = len(e2e_slots) * (sum(I * R for I, R in zip(W["dims"], W["ranks"])) + int(np.prod(W["ranks"]))) * 4
        e2e = {"value": whole_job_rate(len(e2e_slots) * e2e_steps, world, e2e_s), "unit": "decomps/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "step_ms": step_ms,
               "path": f"tucker_server_* request loop, {len(P['slots'])} requests per step, pinned host input and "
                       f"output buffers, host clock around the steps"}
        # the host link that bounds it: one pinned tensor copied to the device, CUDA events around it
        try:
            dev = torch.empty_like(host_in[0], device="cuda")
            rates = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(b.main_s)
                with torch.cuda.stream(b.main_s):
                    dev.copy_(host_in[0], non_blocking=True)
                e1.record(b.main_s)
                b.main_s.synchronize()
                rates.append(host_in[0].numel() * host_in[0].element_size() / (e0.elapsed_time(e1) * 1e-3) / 1e9)
            link = max(rates)
            bound = len(e2e_slots) / ((h2d + d2h) / (link * 1e9))
            e2e["h2d_link_gbs"] = link
            e2e["copy_bound_decomps_per_s"] = bound
            e2e["frac_of_copy_bound"] = e2e["value"] / bound
            # the same steps with the copies alone (every slot's input to the device, host clock
            # around each step): single copies on this host's link now and then take 2.5x their
            # usual time, in a copy loop without any decomposition as well as in the request loop,
            # and this loop meets those stalls over as many steps as the timed ones
            loop_ms = []
            for _ in range(e2e_steps):
                t1 = time.perf_counter()
                with torch.cuda.stream(b.main_s):
                    for h in host_in:
                        dev.copy_(h, non_blocking=True)
                b.main_s.synchronize()
                loop_ms.append(round(1e3 * (time.perf_counter() - t1), 1))
            loop_rate = len(e2e_slots) * e2e_steps / (sum(loop_ms) / 1e3)
            e2e["copy_loop"] = {"decomps_per_s": loop_rate, "step_ms": loop_ms,
                                "what": "the timed steps' host-to-device copies alone, one stream, host clock"}
            e2e["frac_of_copy_loop"] = e2e["value"] / loop_rate
            del dev
        except Exception as exc:  # noqa: BLE001
            e2e["h2d_link_error"] = str(exc)[:200]
        del host_in, houts
    except Exception as exc:  # noqa: BLE001
        e2e = {"value": None, "unit": "decomps/s", "error": str(exc)}

    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_or = len(P["oracle"])
        secs = sum(o["seconds"] for o in P["oracle"].values())
        cpu_baseline = {"value": n_or / secs, "unit": "decomps/s", "cores": cpu_cores(), "kind": "oracle",
                        "sample": f"{n_or} whole {HEADLINE} decompositions ({', '.join(P['oracle'])}) of the first "
                                  f"tensor in {secs:.1f} s, numpy FP64 with its BLAS on all host cores (the same "
                                  f"runs give the oracle's relative errors)"}
    head_line = {p: {"value": r["value"], "ms_per_step": r["ms"] / args.steps, "gpu_launches": r["gpu_launches"],
                     "accuracy": r["accuracy"], "re_within_1e_3_of_oracle": r["re_within_1e_3_of_oracle"],
                     "re_within_1e_5_of_oracle": r["re_within_1e_5_of_oracle"]} for p, r in res.items()}
    del P
    torch.cuda.empty_cache()

    # ---- secondary workloads
    secondary = {}
    if not args.no_secondary:
        for name in ("video1024_range", "cube400", "cube400_related", "quartic96", "fp64cube100"):
            try:
                Wn = WORKLOADS[name]
                Pn, rn = b.workload_line(name, Wn.get("forms", forms), max(3, args.steps // 2))
                okn = [p for p in rn if rn[p]["re_within_1e_3_of_oracle"]] or list(rn)
                hn = max(okn, key=lambda p: rn[p]["value"])
                secondary[name] = {
                    "workload": Wn["desc"], "headline_form": hn, "value": rn[hn]["value"], "unit": "decomps/s",
                    "distinct_tensors": Pn["distinct"], "slots": len(Pn["slots"]),
                    "oracle_decomps_per_s": len(Pn["oracle"]) / Pn["oracle_seconds"],
                    "forms": {p: {"value": r["value"], "ms_per_step": r["ms"] / max(3, args.steps // 2),
                                  "accuracy": r["accuracy"], "re_within_1e_3_of_oracle": r["re_within_1e_3_of_oracle"],
                                  "re_within_1e_5_of_oracle": r["re_within_1e_5_of_oracle"]} for p, r in rn.items()}}
                if name == "cube400":
                    # randomized T-HOSVD (Algorithm 1) of the low-rank tensors in the headline form
                    low = [A for v, A in Pn["slots"] if v["gen"] == "lowrank"]
                    tb = tk.Batch([dict(which="T", A=A, dims=Wn["dims"], ranks=Wn["ranks"], P=Wn["P"], q=1, c=0,
                                        prob="uniform", seed=SEED + k) for k, A in enumerate(low + low)], prec=hn)
                    for _ in range(args.warmup):
                        tb.run(stream=b.main_s, sync=False)
                    tb.run(stream=b.main_s)
                    ts = max(3, args.steps // 4)
                    b.barrier()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(b.main_s)
                    for _ in range(ts):
                        tb.run(stream=b.main_s, sync=False)
                    e1.record(b.main_s)
                    b.main_s.synchronize()
                    b.barrier()
                    secondary["thosvd400"] = {
                        "value": whole_job_rate(2 * len(low) * ts, world, b.max_over_ranks(e0.elapsed_time(e1)) / 1e3),
                        "unit": "decomps/s", "prec": hn,
                        "workload": f"randomized T-HOSVD of {len(low)} distinct 400^3 low-rank tensors (each twice, "
                                    f"different seeds), R=20 P=10 q=1, one tucker_batch_run call per step"}
                    del tb
                del Pn
                torch.cuda.empty_cache()
            except Exception as exc:  # noqa: BLE001
                secondary[name] = {"error": str(exc)[:300]}

    latency = None
    if not args.no_secondary:
        try:
            latency = latency_bench(tk, torch, b.main_s, list(dict.fromkeys([head, "fp32"])))
        except Exception as exc:  # noqa: BLE001
            latency = {"error": str(exc)[:300]}
        try:
            secondary["fusions"] = fusion_bench(tk, torch, b.main_s)
        except Exception as exc:  # noqa: BLE001
            secondary["fusions"] = {"error": str(exc)[:300]}
        try:
            secondary["adaptive_ranks"] = adaptive_bench(tk, torch, list(dict.fromkeys([head, "fp32"])))
        except Exception as exc:  # noqa: BLE001
            secondary["adaptive_ranks"] = {"error": str(exc)[:300]}

    serving = None
    if not args.no_serving:
        try:
            specs = serving_specs()
            serving = {p: serving_bench(tk, torch, specs, p) for p in dict.fromkeys([head, "fp32"]) if p in forms}
            serving["stream"] = (f"{len(specs)} randomized ST-HOSVD requests (P=5, q=1), order 3 or 4, every extent "
                                 f"U{{32..256}}, ranks U{{4..32}}, low-rank + 1e-2 noise FP32 (order 4 up to 17 GB); "
                                 f"server budget {SERVE_BUDGET >> 30} GB, 16 streams; inputs generated on the device "
                                 f"in groups of at most {SERVE_RESIDENT >> 30} GB before each group (untimed); "
                                 f"saturation = each group at once; latency under Poisson arrivals at 0.7x the "
                                 f"saturation rate within each group")
        except Exception as exc:  # noqa: BLE001
            serving = {"error": str(exc)[:300]}
    clk = b.clocks.stop()

    line = {"metric": "decomps/s", "value": res[head]["value"], "unit": "decomps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res[head]["ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "baseline_metric": BASELINE_METRIC,
            "config": {"workload": W["desc"], "headline_form": head, "slots_per_step": len(W["variants"]) * W["copies"],
                       "tensor_bytes": int(np.prod(W["dims"])) * 4,
                       "l2": "inputs larger than L2 (2.15 GB per tensor), no flush",
                       "parallelism": "replicas (each rank decomposes its own batch)" if world > 1 else "single GPU",
                       "execution": f"tucker_batch_run per step: one CUDA graph (captured by the library on its "
                                    f"first run, replayed after) of {len(W['variants']) * W['copies']} "
                                    f"decompositions on as many streams, distinct inputs (one tensor per slot)",
                       "headline_rule": "fastest form whose relative error is within 1e-3 of the FP64 oracle's on "
                                        "every variant (oracle on the same bytes, this run)",
                       "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS")},
            "e2e": e2e, "gpu_launches": res[head]["gpu_launches"], "roofline": roofline, "kernels": kernels,
            "sketch_hbm_gbs": achieved_gbs,
            "forms": head_line,
            "secondary": secondary,
            "latency": latency,
            "serving": serving,
            "autotune": tk.autotune_entries(),
            "clocks": clk}
    if cpu_baseline:
        line["cpu_baseline"] = cpu_baseline
        line["cpu_baseline_1thread"] = oracle_one_thread(HEADLINE, W["variants"][0]["name"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
