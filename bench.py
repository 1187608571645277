#!/usr/bin/env python3
"""Benchmark of the MaxSAT gradient engine: fwd+bwd literal-evals per second.

One benchmark step is one iteration of Algorithm 1 for every restart of the
workload: the clause pass (relaxed values, exact unsat cost, loss partials)
and the variable pass (gradient over the transposed CSR, Adam, best
assignment).  Work = nnz * B literal-evaluations per step (each literal of
each restart is gathered forward and scattered backward once).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl ours|reference]

--impl reference times the CPU oracle on the same instance (a bounded
sample per step).  Under torchrun every rank runs its own replica of the
workload (the restarts and instances are independent; no collective on the
data path); rank 0 prints one JSON line.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import ordering, pigeonhole, random_partial, serving_stream, uniform_ksat, zipf_weighted  # noqa: E402

L2_BYTES = 129 * 2 ** 20

WORKLOADS = {
    # name: (generator, restarts, description)
    "ksat3_n5000_m21500_b256": (lambda: uniform_ksat(5000, 21500, 3, seed=0), 256,
                                "uniform random 3-SAT, n=5000, m=21500 (seed 0), B=256 restarts, x from seed 1; "
                                "each step also evaluates the rounded +-1 batch on the tensor cores"),
    "ksat3_n1000000_m4300000_b16": (lambda: uniform_ksat(1000000, 4300000, 3, seed=0), 16,
                                    "uniform random 3-SAT, n=1e6, m=4.3e6 (seed 0), B=16 restarts"),
    "zipf_n200000_m1000000_weighted_b1": (lambda: zipf_weighted(200000, 1000000, seed=0), 1,
                                          "weighted MaxSAT, n=2e5, m=1e6, lengths 2+Geom(1/3)<=20, Zipf(1.2) variables, weights 1..1000, B=1"),
    "ksat3_n50_m215_b1": (lambda: uniform_ksat(50, 215, 3, seed=0), 1,
                          "uniform random 3-SAT, n=50, m=215 (seed 0), B=1"),
}
# the line's value: the largest configuration on one GPU, 3-SAT n=1e6, B=16
DEFAULT_WORKLOAD = "ksat3_n1000000_m4300000_b16"
# measured beside it: batched restarts with the tensor-core evaluation
DENSE_WORKLOAD = "ksat3_n5000_m21500_b256"
# the request stream of the serving measurement: k in {3,4,5}, n log-uniform
# in [100, 50000], ratio U[4.0, 4.6] scaled to each k's threshold, Poisson
# arrivals; each request takes SERVE_STEPS steps with SERVE_RESTARTS restarts
SERVING = "serving_k345_b8"
SERVE_STREAM_LEN = 10000
SERVE_STEPS = 1000
SERVE_RESTARTS = 8
# cost-vs-time curves of Algorithm 1 with its time limit on the structured
# families of Table 2 (pigeonhole PHP and ordering GT, optimum cost 1)
STRUCTURED = "structured_cost_time"
# the rows after the hot path: the loss normalisers of the ablation on the
# default instance, steps to the best cost, the quick f_j > 0 reading against
# the exact test, and a partial MaxSAT instance
NEXT_ROWS = "next_rows_loss_partial"
# workloads whose step also runs the dense tensor-core evaluation of the rounded batch
DENSE_EVAL = {"ksat3_n5000_m21500_b256"}
LR = 1e-4


def algorithmic_bytes(cnf, B):
    """Minimum bytes each pass must move per launch.  Clause pass: the
    literal stream (4 nnz), each t value once (4 n B), the unsat bits
    (m B / 8), plus clause offsets when lengths differ and the weights.
    Variable pass: occurrence offsets and lists (4 (n+1) + 4 nnz), the unsat
    bits, x, m and v read and written (24 n B) and t written (4 n B)."""
    n, m, nnz = cnf.n, cnf.m, cnf.nnz
    lens = np.diff(cnf.off)
    uniform = m > 0 and bool(np.all(lens == lens[0]))
    fwd = 4 * nnz + 4 * n * B + m * B / 8.0
    if not uniform:
        fwd += 4 * (m + 1)
    if cnf.weights is not None:
        fwd += 8 * m
    bwd = 4 * (n + 1) + 4 * nnz + m * B / 8.0 + 24 * n * B + 4 * n * B
    return {"forward": fwd, "backward": bwd}


# nominal dense tensor rates of the part: fp4 13.5 and bf16 2.25 PFLOP/s
FP4_PER_BF16 = 13.5 / 2.25


def measured_peaks():
    """(HBM GB/s, source), (fp4 dense TFLOP/s, source): the copy bandwidth and
    the bf16 GEMM rate measured on these GPUs, fp4 (the dense evaluator's
    block-scaled e2m1 MMA) taken as bf16 times the nominal fp4:bf16 ratio."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return ((float(d["hbm_gbs"]), "measured"),
                (FP4_PER_BF16 * float(d["bf16_tflops"]), "measured bf16 x 6 (nominal fp4:bf16 ratio)"))
    return (6800.0, "fallback"), (FP4_PER_BF16 * 1900.0, "fallback bf16 x 6 (nominal fp4:bf16 ratio)")


def dense_roofline(pkg, m, n, B, avg_s, peak_gbs, tc_peak, tc_kind):
    """Both bounds of one dense evaluation: the packed clause matrix W^T
    (m x n e2m1 codes, half a byte each), the packed batch (B x n) and the
    per-clause target and weight (8 bytes) read once, against HBM; 2 m n B
    flops against the fp4 tensor peak.  The binding one is reported, with
    the MMA rate of the evaluator's own instruction shape measured live
    beside it."""
    flops = 2.0 * m * n * B
    nbytes = m * n / 2.0 + B * n / 2.0 + 8.0 * m
    tf = flops / avg_s / 1e12
    gbs = nbytes / avg_s / 1e9
    t_tc, t_hbm = flops / (tc_peak * 1e12), nbytes / (peak_gbs * 1e9)
    ntile = min(256, (B + 15) // 16 * 16)
    inst = pkg.dense_mma_rate(ntile, 4096)
    ent = {"avg_us": 1e6 * avg_s, "flops": flops, "tflops": tf, "bytes": nbytes, "gbs": gbs,
           "tensor_frac": tf / tc_peak, "hbm_frac": gbs / peak_gbs, "peak_tflops": tc_peak,
           "peak_source": tc_kind, "peak_gbs": peak_gbs,
           "instruction_peak_tflops": inst, "instruction_frac": tf / inst,
           "instruction_peak_source": f"msat_dense_mma_rate: kind::mxf4 M=128 N={ntile} K=64 issued back to "
                                      "back on every SM, operands resident in shared memory"}
    if t_tc >= t_hbm:
        ent.update(bound="tensor", frac=tf / tc_peak)
    else:
        ent.update(bound="hbm", frac=gbs / peak_gbs)
    return ent


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                 power=float(parts[3]) if parts[3] not in ("[N/A]", "N/A") else None,
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
            except ValueError:
                continue
        if not rows:
            return None
        loaded = [r for r in rows if r["power"] is not None and r["power"] > 250.0] or rows
        reasons = set()
        for r in loaded:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in loaded),
                "sm_max_mhz": max(r["smax"] for r in rows), "reasons": sorted(reasons),
                "samples": len(rows), "samples_under_load": len(loaded)}


def cpu_oracle_rate(cnf, B, budget_s=12.0, max_steps=200):
    """Literal-evals/s of the FP32-mode oracle (Algorithm 1 on one host thread)."""
    from oracle import oracle
    oracle.build()
    t = time.perf_counter()
    oracle.solve(cnf, B, 1, 1, mode=oracle.MODE_F32, want_hist=False, want_x=False)
    one = max(time.perf_counter() - t, 1e-4)
    steps = int(max(1, min(max_steps, budget_s / one)))
    t = time.perf_counter()
    oracle.solve(cnf, B, 1, steps, mode=oracle.MODE_F32, want_hist=False, want_x=False)
    dt = time.perf_counter() - t
    # solve() also evaluates x_0 .. x_steps: steps updates + one extra evaluation
    return cnf.nnz * B * steps / dt, steps, dt


def host_cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_oracle_rate_threads(cnf, B, threads, budget_s=12.0, max_steps=200):
    """Literal-evals/s of the FP32-mode oracle on `threads` host threads:
    restarts are independent, so the B restarts are split into `threads`
    groups (or, when B < threads, `threads` independent copies of the
    one-restart problem run side by side), each solved by its own oracle
    call on its own thread (the C oracle runs without the interpreter lock).
    The oracle's arithmetic is untouched; only whole restarts are spread."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle
    oracle.build()
    per = max(1, B // threads)
    t = time.perf_counter()
    oracle.solve(cnf, per, 1, 1, mode=oracle.MODE_F32, want_hist=False, want_x=False)
    one = max(time.perf_counter() - t, 1e-4)
    steps = int(max(1, min(max_steps, budget_s / one)))

    def job(k):
        oracle.solve(cnf, per, 1 + k, steps, mode=oracle.MODE_F32, want_hist=False, want_x=False)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        t = time.perf_counter()
        list(ex.map(job, range(threads)))
        dt = time.perf_counter() - t
    return cnf.nnz * per * threads * steps / dt, steps, dt, per


def cpu_baseline_entry(cnf, B):
    """The oracle as it stands, timed on the host's cores: one thread, and
    all of them (nproc) over restarts."""
    rate, csteps, cdt = cpu_oracle_rate(cnf, B)
    nproc = os.cpu_count() or 1
    mt = None
    if nproc > 1:
        mrate, msteps, mdt, per = cpu_oracle_rate_threads(cnf, B, nproc)
        mt = {"value": mrate, "unit": "literal-evals/s", "cores": nproc,
              "sample": f"{nproc} threads, each {msteps} Algorithm 1 steps of the FP32-mode C oracle "
                        f"on the full instance with {per} restart(s) ({mdt:.1f} s)"}
    return {"value": rate, "unit": "literal-evals/s", "cores": 1, "kind": "oracle",
            "sample": f"{csteps} Algorithm 1 steps of the FP32-mode C oracle on the full "
                      f"instance, all {B} restarts, one host thread ({cdt:.1f} s)",
            "cpu_model": host_cpu_model(), "host_cores": nproc, "all_cores": mt}


def parse_shape(text):
    """--shape FWD_VW:STAGE_VW:LIGHT_ROWS (0 = automatic) as Solver keywords."""
    if not text:
        return None
    a, b, c = (int(v) for v in text.split(":"))
    return {"fwd_vw": a, "stage_vw": b, "light_rows": c}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference_serving(args):
    """The oracle on the serving stream: each sampled request solved with a
    reduced step count, its time scaled to the request's full step count
    (the per-step work of Algorithm 1 is constant)."""
    from oracle import oracle
    oracle.build()
    B, steps, probe = SERVE_RESTARTS, SERVE_STEPS, 10
    reqs = serving_stream(SERVE_STREAM_LEN, rate_per_s=args.serve_rate, seed=0)
    budget = 20.0
    spent, est, used = 0.0, 0.0, 0
    for r in reqs:
        if spent > budget:
            break
        c = r.instance()
        t = time.perf_counter()
        oracle.solve(c, B, r.seed, probe, mode=oracle.MODE_F32, want_hist=False, want_x=False)
        dt = time.perf_counter() - t
        spent += dt
        est += dt * (steps + 1) / (probe + 1)
        used += 1
    value = used / est
    sample = (f"the first {used} requests of the serving stream, {probe} of the {steps} steps each "
              f"run by the FP32-mode C oracle on one host thread, time scaled by {steps + 1}/{probe + 1}")
    line = {
        "impl": "reference", "metric": "instances/s", "value": value, "unit": "instances/s",
        "n_gpus": 1, "steps": steps, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": SERVING, "restarts": B, "steps_per_request": steps},
        "cpu_baseline": {"value": value, "unit": "instances/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "instances/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == SERVING:
        return run_reference_serving(args)
    if args.workload == STRUCTURED:
        print(json.dumps({"impl": "reference", "unavailable": "the cost-vs-time curves have no oracle arm: "
                          "the oracle has no wall-clock limit"}), flush=True)
        return 0
    if args.workload == NEXT_ROWS:
        print(json.dumps({"impl": "reference", "unavailable": "the ablation and partial-MaxSAT runs have no "
                          "oracle arm: the oracle pins these rows in the tests"}), flush=True)
        return 0
    gen, B, desc = WORKLOADS[args.workload]
    cnf = gen()
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle
    oracle.build()
    # restarts are independent: every host core solves its own group of
    # restarts (its own oracle call on its own thread; the C oracle runs
    # without the interpreter lock), each step a bounded sample of the B
    # restarts so the whole run stays within a few minutes; the metric is
    # per literal-evaluation
    threads = os.cpu_count() or 1
    t = time.perf_counter()
    oracle.solve(cnf, 1, 1, 1, mode=oracle.MODE_F32, want_hist=False, want_x=False)
    per_restart = max(time.perf_counter() - t, 1e-4)
    per = int(max(1, min(max(1, B // threads), 20.0 / max(1, args.steps + args.warmup) / per_restart)))

    def run(pool, steps):
        list(pool.map(lambda k: oracle.solve(cnf, per, 1 + k, steps, mode=oracle.MODE_F32, want_hist=False,
                                             want_x=False), range(threads)))

    with ThreadPoolExecutor(max_workers=threads) as pool:
        run(pool, args.warmup)  # untimed
        t = time.perf_counter()
        run(pool, args.steps)   # K steps of Algorithm 1 on every thread at once
        total = time.perf_counter() - t
    value = cnf.nnz * per * threads * args.steps / total
    sample = (f"one call of {args.steps} Algorithm 1 steps (plus the final evaluation) for {per} restart(s) "
              f"on each of {threads} host threads at once ({per * threads} restarts; the workload has {B}), "
              f"FP32-mode C oracle, after an untimed call of {args.warmup} steps")
    line = {
        "impl": "reference", "metric": "fwd+bwd literal-evals/s", "value": value,
        "unit": "literal-evals/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": cnf.n, "m": cnf.m,
                   "nnz": cnf.nnz, "restarts": B, "restarts_per_step_sampled": per * threads},
        "cpu_baseline": {"value": value, "unit": "literal-evals/s", "cores": threads, "kind": "oracle",
                         "sample": sample, "cpu_model": host_cpu_model()},
        "e2e": {"value": value, "unit": "literal-evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_workload(pkg, args, workload, ws, rank, with_cpu=True, with_e2e=True):
    """The benchmark line of one workload: K device-timed steps (graph
    replay), per-kernel roofline, end-to-end run through the public calls
    and the oracle's CPU baseline."""
    import torch
    dev = torch.cuda.current_device()
    gen, B, desc = WORKLOADS[workload]
    cnf = gen()
    nnz = cnf.nnz
    work_per_step = nnz * B
    abytes = algorithmic_bytes(cnf, B)
    working_set = sum(abytes.values())
    flush = working_set < 2 * L2_BYTES
    flush_buf = torch.empty(64 * 2 ** 20, dtype=torch.float32, device="cuda") if flush else None

    # launch shapes from the library's autotuner (they never change a result
    # bit), or fixed by --shape (profiling captures skip the tuner's launches)
    shape = parse_shape(args.shape)
    solver = pkg.Solver.from_cnf(cnf, restarts=B, seed_x=1, lr=LR, tune=shape is None,
                                 f_mode=args.f_mode, **(shape or {}))
    stream = torch.cuda.current_stream()
    dense = workload in DENSE_EVAL
    dense_cost = torch.empty(B, dtype=torch.int64, device="cuda")
    # small instances run every step of a call in one single-CTA launch:
    # time one call of K steps (per-pass timing would force the per-pass
    # kernels)
    small = bool(solver.info()["small_kernel"]) and not dense

    def one_step():
        solver.step_async(1, final_eval=False)
        if dense:
            solver.evaluate_x("dense", out=dense_cost)

    # warm-up, then a short clock-settling run, both untimed
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    t_settle = time.perf_counter()
    while time.perf_counter() - t_settle < 0.5:
        for _ in range(20):
            one_step()
        torch.cuda.synchronize()

    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if not small:
        solver.profile(True)
        solver.profile_read(reset=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    if small:
        if flush:
            flush_buf.zero_()
        ev_s[0].record(stream)
        solver.step_async(args.steps, final_eval=False)
        ev_e[0].record(stream)
    else:
        for k in range(args.steps):
            if flush:
                flush_buf.zero_()
            ev_s[k].record(stream)
            one_step()
            ev_e[k].record(stream)
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    if ws > 1:
        torch.distributed.barrier()

    def graph_replay_ms():
        """The same step replayed from a CUDA graph of its launches (no host
        gaps between them): K timed replays, L2 flushed before each."""
        cap = torch.cuda.Stream()
        try:
            solver.set_stream(cap)
            with torch.cuda.stream(cap):
                for _ in range(2):
                    one_step()
            cap.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                one_step()
        finally:
            solver.set_stream(stream)
        torch.cuda.synchronize()
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        es = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ee = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if ws > 1:
            torch.distributed.barrier()
        for k in range(args.steps):
            if flush:
                flush_buf.zero_()
            es[k].record(stream)
            g.replay()
            ee[k].record(stream)
        torch.cuda.synchronize()
        return float(sum(es[k].elapsed_time(ee[k]) for k in range(args.steps)))

    plain_ms, graph_err = None, None
    if small:
        dev_ms = float(ev_s[0].elapsed_time(ev_e[0]))
        prof = {"forward": (0, 0.0), "backward": (0, 0.0), "evaluate": (0, 0.0), "other": (1, dev_ms)}
    else:
        prof = solver.profile_read(reset=True)
        solver.profile(False)
        step_ms = [ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)]
        plain_ms = dev_ms = float(sum(step_ms))
        try:
            dev_ms = graph_replay_ms()
        except Exception as ex:  # keep the plain-launch timing
            graph_err = repr(ex)[:200]
    clk = clocks.stop()
    from paper_2402_03640_gb300 import replicas
    t_max, units = replicas.combine(dev_ms, float(work_per_step * args.steps),
                                    device="cuda" if ws > 1 else None)
    value = units / (t_max / 1e3)

    # roofline of the dominant kernel, from the events around each launch
    (peak, peak_kind), (tc_peak, tc_kind) = measured_peaks()
    per_kernel = {}
    for kind in ("forward", "backward"):
        launches, ms = prof[kind]
        if launches:
            avg = ms / launches
            per_kernel[kind] = {"launches": launches, "avg_us": 1e3 * avg, "bound": "hbm",
                                "bytes": abytes[kind], "gbs": abytes[kind] / (avg / 1e3) / 1e9,
                                "frac": abytes[kind] / (avg / 1e3) / 1e9 / peak}
    if small:
        per_step = dev_ms / args.steps
        by = abytes["forward"] + abytes["backward"]
        per_kernel["small_steps"] = {"launches": 1, "steps_per_launch": args.steps,
                                     "avg_us": 1e3 * per_step, "bound": "hbm", "bytes": by,
                                     "gbs": by / (per_step / 1e3) / 1e9,
                                     "frac": by / (per_step / 1e3) / 1e9 / peak}
        abytes["small_steps"] = by
    if dense and prof["evaluate"][0]:
        launches, ms = prof["evaluate"]
        per_kernel["dense_eval"] = dict(launches=launches, **dense_roofline(
            pkg, cnf.m, cnf.n, B, ms / launches / 1e3, peak, tc_peak, tc_kind))
        abytes["dense_eval"] = per_kernel["dense_eval"]["bytes"]
    dom = max(per_kernel, key=lambda k: per_kernel[k]["avg_us"] * per_kernel[k]["launches"])
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            tr = json.load(f)
        ent = tr.get(workload, {}).get(dom)
        if ent and ent.get("kernel_hash") == kernel_hash(dom):
            traffic = ent["bytes_per_launch"]
    if per_kernel[dom]["bound"] == "tensor":
        ach = per_kernel[dom]["tflops"]
        roofline = {"bound": "tensor", "achieved": ach, "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": ach / tc_peak, "traffic": traffic, "kernel": dom,
                    "peak_source": tc_kind, "algorithmic_flops_per_launch": per_kernel[dom]["flops"]}
        if dom == "dense_eval":
            roofline["instruction_peak"] = per_kernel[dom]["instruction_peak_tflops"]
    else:
        ach = per_kernel[dom]["gbs"]
        roofline = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "traffic": traffic, "kernel": dom,
                    "peak_source": f"{peak_kind} hbm_gbs (copy bandwidth)",
                    "algorithmic_bytes_per_launch": abytes[dom]}

    # end to end through the public API with host buffers: upload the CNF
    # from host memory (context creation inside the timed region), then per
    # step the calls a user makes for the work of the timed step -- the
    # optimizer step replayed from the library's CUDA graph and, on the
    # default workload, the tensor-core evaluation of the new x -- and the
    # step's B costs read back into pinned host memory
    e2e = measure_e2e(pkg, cnf, B, args, dense, ws, dict(solver.tuning or shape or {})) if with_e2e else None

    cpu = None
    if rank == 0 and with_cpu and not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(cnf, B)

    launches = prof["forward"][0] + prof["backward"][0] + prof["evaluate"][0] + prof["other"][0]
    info = solver.info()
    _, cost = solver.step(0, want_loss=False)
    dense_ok = None
    if dense:
        dense_ok = bool(np.array_equal(solver.evaluate_x("dense").cpu().numpy(), cost))
        solver.check()
    line = {
        "metric": "fwd+bwd literal-evals/s", "value": value, "unit": "literal-evals/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "ms_per_step_plain_launches": None if plain_ms is None else plain_ms / args.steps,
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload, "description": desc, "n": cnf.n, "m": cnf.m,
                   "nnz": nnz, "restarts": B, "lr": LR,
                   "l2": ("flushed (256 MiB write) before the timed call, whose K steps run in one "
                          "single-CTA launch with the state in shared memory" if small else
                          "flushed (256 MiB write) before every timed step" if flush
                          else "working set larger than L2"),
                   "route": "single-CTA kernel" if small else "per-pass kernels",
                   "launch": ("one launch of K steps" if small else
                              "each step replayed from a CUDA graph of its launches" if graph_err is None
                              else "plain launches (graph capture failed: %s)" % graph_err),
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "f_mode": args.f_mode,
                   "n_heavy": info["n_heavy"]},
        "roofline": roofline,
        "kernels": per_kernel,
        "cpu_baseline": cpu,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": launches,
        "tuned_shape": (solver.tuning and {k: solver.tuning[k] for k in ("fwd_vw", "stage_vw", "light_rows")})
                       or (shape and dict(shape, fixed_by="--shape")),
        "wall_s_timed": wall1 - wall0,
        "final_cost_min": int(cost.min()),
        "dense_eval_matches_sparse": dense_ok,
    }
    solver.close()
    return line


def measure_e2e(pkg, cnf, B, args, dense, ws, shape_kw):
    """End to end through the public API with host buffers: upload the CNF
    from host memory (context creation inside the timed region), then per
    step the calls a user makes for the work of the timed step -- the
    optimizer step replayed from the library's CUDA graph and, on the dense
    evaluation workload, the tensor-core evaluation of the new x -- and the
    step's B costs read back into host memory."""
    import torch
    from paper_2402_03640_gb300 import replicas
    work_per_step = cnf.nnz * B
    torch.cuda.synchronize()
    e2e_steps = args.steps
    h2d = cnf.off.nbytes + cnf.lits.nbytes + (0 if cnf.weights is None else cnf.weights.nbytes)
    hcost = torch.empty(B, dtype=torch.int64).pin_memory()
    dcost = torch.empty(B, dtype=torch.int64, device="cuda")
    t0 = time.perf_counter()
    shape_kw = {k: shape_kw[k] for k in ("fwd_vw", "stage_vw", "light_rows") if k in shape_kw}
    s2 = pkg.Solver.from_cnf(cnf, restarts=B, seed_x=1, lr=LR, f_mode=args.f_mode, **shape_kw)
    t_create = time.perf_counter() - t0
    for _ in range(e2e_steps):
        if dense:  # the final sparse evaluation is replaced by the dense one
            s2.step_async(1, final_eval=False, graph=True)
            s2.evaluate_x("dense", out=dcost)
            hcost.copy_(dcost, non_blocking=True)
            torch.cuda.current_stream().synchronize()
        else:
            s2.step(1, want_loss=False, graph=True)
    t1 = time.perf_counter()
    s2.close()
    e_max, e_units = replicas.combine(t1 - t0, float(work_per_step * e2e_steps),
                                      device="cuda" if ws > 1 else None)
    e2e_value = e_units / e_max
    return {"value": e2e_value, "unit": "literal-evals/s", "h2d_bytes_per_step": h2d / e2e_steps,
            "d2h_bytes_per_step": B * 8, "steps": e2e_steps, "create_ms": 1e3 * t_create,
            "note": "msat_create from host arrays once inside the timed region (create_ms), then "
                    "per step " +
                    ("msat_step(1) replayed from the library's CUDA graph without its final "
                     "evaluation, msat_evaluate_x on the tensor cores, and the B costs copied "
                     "to pinned host memory" if dense else
                     "msat_step(1) replayed from the library's CUDA graph with the B costs of "
                     "its final evaluation copied to host memory")}


def dense_steady_state(pkg, sms=152, waves=8):
    """The tensor-core evaluator's own rate with whole waves of tiles: 3-SAT
    with n = 5120 (20 k-steps of 256 variables a tile) and 128 * sms * waves clauses, 256
    assignments (one assignment tile), so every CTA of the one-per-SM grid
    takes `waves` whole tiles and no tile is split; the packed clause matrix
    (50 MB per wave of tiles, 400 MB in all) is streamed from HBM.  Ten timed
    launches after three untimed ones; both bounds as in dense_roofline."""
    import torch
    n, B = 5120, 256
    m = 128 * sms * waves
    cnf = uniform_ksat(n, m, 3, seed=3)
    out = torch.empty(B, dtype=torch.int64, device="cuda")
    with pkg.Solver.from_cnf(cnf, restarts=B, seed_x=1, lr=LR) as s:
        for _ in range(3):
            s.evaluate_x("dense", out=out)
        torch.cuda.synchronize()
        s.profile(True)
        s.profile_read(reset=True)
        for _ in range(10):
            s.evaluate_x("dense", out=out)
        torch.cuda.synchronize()
        prof = s.profile_read(reset=True)
        s.profile(False)
        s.check()
    launches, ms = prof["evaluate"]
    (peak_gbs, _), (tc_peak, tc_kind) = measured_peaks()
    ent = {"workload": f"uniform 3-SAT n={n}, m={m} (seed 3), {B} assignments: {waves} waves of whole "
                       f"128 x 256 tiles on {sms} SMs, no split tile", "launches": launches}
    ent.update(dense_roofline(pkg, m, n, B, ms / launches / 1e3, peak_gbs, tc_peak, tc_kind))
    return ent


def other_configs(pkg, args, rank):
    """The plain single instance (3-SAT n=50, m=215, 1000 steps) and the
    weighted Zipf instance (n=2e5, m=1e6, weights 1..1000, 500 steps), B = 1,
    x from seed 1, lr 1e-4: final and best (weighted) unsat cost and the
    device time per step.  Their cpu_baseline leg runs the FP32-mode oracle
    on the same configuration (one host thread) and records its time and its
    costs, which the GPU's must equal."""
    import torch
    out = {}
    for name, steps in (("ksat3_n50_m215_b1", 1000), ("zipf_n200000_m1000000_weighted_b1", 500)):
        gen, B, desc = WORKLOADS[name]
        cnf = gen()
        with pkg.Solver.from_cnf(cnf, restarts=B, seed_x=1, lr=LR) as s:
            s.step(0, want_loss=False)
            torch.cuda.synchronize()
            stream = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step_async(steps)  # Algorithm 1: `steps` iterations, then the evaluation of x_steps
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            _, cost = s.step(0, want_loss=False)
            _, best = s.best()
            route = "single-CTA kernel" if s.info()["small_kernel"] else "per-pass kernels"
        ent = {"description": desc, "n": cnf.n, "m": cnf.m, "nnz": cnf.nnz, "restarts": B, "steps": steps,
               "lr": LR, "route": route, "ms": ms, "us_per_step": 1e3 * ms / steps,
               "literal_evals_per_s": cnf.nnz * B * steps / (ms / 1e3),
               "final_cost": int(cost[0]), "best_cost": int(best[0]),
               "cost_dtype": "int64 (weighted)" if cnf.weights is not None else "int64 (count)"}
        if rank == 0 and not args.no_cpu_baseline:
            from oracle import oracle
            oracle.build()
            t = time.perf_counter()
            ref = oracle.solve(cnf, B, 1, steps, mode=oracle.MODE_F32, lr=LR, want_x=False)
            dt = time.perf_counter() - t
            ent["cpu_baseline"] = {"value": cnf.nnz * B * steps / dt, "unit": "literal-evals/s", "cores": 1,
                                   "kind": "oracle", "seconds": dt,
                                   "sample": f"the whole run ({steps} steps, FP32-mode C oracle, one host thread)",
                                   "final_cost": int(ref["cost_hist"][-1][0]), "best_cost": int(ref["best_cost"][0])}
            ent["costs_equal_oracle"] = (ent["final_cost"] == ent["cpu_baseline"]["final_cost"]
                                         and ent["best_cost"] == ent["cpu_baseline"]["best_cost"])
        out[name] = ent
    return out


def run_ours(args):
    import torch
    import paper_2402_03640_gb300 as pkg
    from paper_2402_03640_gb300 import build as pkg_build

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    pkg_build.build()
    pkg.load()
    line = measure_workload(pkg, args, args.workload, ws, rank)
    if args.workload == DEFAULT_WORKLOAD and not args.no_extras:
        # the other configurations, each measured on its own (not part of value)
        dense_line = measure_workload(pkg, args, DENSE_WORKLOAD, ws, rank, with_cpu=False, with_e2e=False)
        line["dense_eval_workload"] = {k: dense_line[k] for k in (
            "value", "unit", "ms_per_step", "ms_per_step_plain_launches", "config", "roofline", "kernels",
            "dense_eval_matches_sparse", "tuned_shape", "clocks")}
        import torch
        line["dense_eval_workload"]["steady_state"] = dense_steady_state(
            pkg, sms=torch.cuda.get_device_properties(0).multi_processor_count)
        line["configs"] = other_configs(pkg, args, rank)
        if args.serve_requests > 0:
            line["serving"] = serve_compare(pkg, args.serve_requests, args.serve_rate, rank=rank, world=ws)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def _pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    i = min(len(xs) - 1, max(0, int(math.ceil(q / 100.0 * len(xs))) - 1))
    return xs[i]


def serve_compare(pkg, count, rate, steps=SERVE_STEPS, B=SERVE_RESTARTS, lr=LR, rank=0, world=1):
    """The first `count` requests of the serving stream, submitted on their
    Poisson arrival schedule (a) to the continuous-batching server and (b) to
    the plain loop that solves one instance at a time (msat_create, msat_step,
    msat_best, msat_destroy).  Latency runs from a request's arrival to its
    result on the host; instances/s = requests / (last result - first arrival)."""
    from paper_2402_03640_gb300 import replicas
    # under N replicas rank r serves every N-th of the first N*count requests
    reqs = replicas.shard(serving_stream(SERVE_STREAM_LEN, rate_per_s=rate * world, seed=0)[:count * world],
                          rank, world)
    cnfs = [r.instance() for r in reqs]
    warm = uniform_ksat(300, 1290, 3, seed=123)

    def pace(t0, r, stretch=1.0):
        d = t0 + r.arrival_s * stretch - time.perf_counter()
        if d > 0:
            time.sleep(d)

    def served_pass(stretch):
        """The requests through the server with their arrival times scaled by
        `stretch` (a Poisson stream at rate / stretch)."""
        with pkg.Server(restarts=B, lr=lr) as srv:
            srv.wait(srv.submit(warm, 20, seed_x=1))
            t0 = time.perf_counter()
            sub, tickets = [], []
            for r, c in zip(reqs, cnfs):
                pace(t0, r, stretch)
                sub.append(time.perf_counter())
                tickets.append(srv.submit(c, steps, seed_x=r.seed))
            res = [srv.wait(t, 3600.0) for t in tickets]
            st = srv.stats()
        done = [sub[i] + res[i]["latency_ms"] / 1e3 for i in range(count)]
        lat = [done[i] - (t0 + reqs[i].arrival_s * stretch) for i in range(count)]
        return res, lat, max(done) - t0, st

    # (a) served: the burst at the stated rate measures the capacity
    served, lat_a, span_a, st = served_pass(1.0)
    # (a') served at half that capacity: the latency of a sustainable load
    cap = count / span_a
    stretch = max(1.0, rate / (0.5 * cap))
    _, lat_h, span_h, st_h = served_pass(stretch)

    # (b) one instance at a time
    with pkg.Solver.from_cnf(warm, restarts=B, seed_x=1, lr=lr) as s:
        s.step(20, want_loss=False, want_cost=False)
    t0 = time.perf_counter()
    done_b, alone = [], []
    for r, c in zip(reqs, cnfs):
        pace(t0, r)
        with pkg.Solver.from_cnf(c, restarts=B, seed_x=r.seed, lr=lr) as s:
            s.step(steps, want_loss=False, want_cost=False)
            _, best = s.best()
        done_b.append(time.perf_counter())
        alone.append(best)
    lat_b = [done_b[i] - (t0 + reqs[i].arrival_s) for i in range(count)]
    span_b = max(done_b) - t0

    equal = all(np.array_equal(served[i]["best_costs"], alone[i]) for i in range(count))
    lit_evals = sum(c.nnz for c in cnfs) * B * steps
    h2d = sum(c.off.nbytes + c.lits.nbytes + (0 if c.weights is None else c.weights.nbytes) for c in cnfs)
    d2h = sum(B * 8 + c.n for c in cnfs)
    ks = [r.k for r in reqs]
    # whole job: all ranks' requests over the slowest rank's makespan
    _, tot = replicas.combine(0.0, count, device="cuda" if world > 1 else None)
    span_a, _ = replicas.combine(span_a, 0.0, device="cuda" if world > 1 else None)
    span_b, _ = replicas.combine(span_b, 0.0, device="cuda" if world > 1 else None)
    count_all = int(tot)
    return {
        "instances_per_s": count_all / span_a,
        "p50_ms": 1e3 * _pct(lat_a, 50), "p99_ms": 1e3 * _pct(lat_a, 99),
        "one_at_a_time": {"instances_per_s": count_all / span_b, "p50_ms": 1e3 * _pct(lat_b, 50),
                          "p99_ms": 1e3 * _pct(lat_b, 99)},
        "at_half_capacity": {"arrival_rate_per_s": rate * world / stretch,
                             "instances_per_s": count_all / span_h,
                             "p50_ms": 1e3 * _pct(lat_h, 50), "p99_ms": 1e3 * _pct(lat_h, 99),
                             "peak_running": st_h["peak_running"]},
        "small_direct": st["small_direct"],
        "speedup_vs_one_at_a_time": span_b / span_a,
        "final_costs_equal": bool(equal),
        "mean_best_cost": float(np.mean([x["best_cost"] for x in served])),
        "served_literal_evals_per_s": lit_evals * world / span_a,
        "peak_running": st["peak_running"], "graph_captures": st["graph_captures"],
        "requests": count_all, "requests_per_rank": count, "arrival_rate_per_s": rate * world,
        "steps": steps, "restarts": B, "lr": lr,
        "k_counts": {str(k): ks.count(k) for k in (3, 4, 5)},
        "n_range": [min(r.n for r in reqs), max(r.n for r in reqs)],
        "h2d_bytes_per_request": h2d / count, "d2h_bytes_per_request": d2h / count,
        "sample": f"the first {count} of a {SERVE_STREAM_LEN}-request stream (seed 0): k uniform in "
                  "{3,4,5}, n log-uniform in [100, 50000], m/n uniform in [4.0, 4.6] scaled by "
                  "alpha_k/alpha_3, Poisson arrivals",
    }


def run_structured(args):
    import torch
    import paper_2402_03640_gb300 as pkg
    from paper_2402_03640_gb300 import build as pkg_build

    ws, rank, _ = dist_env()
    torch.cuda.set_device(0 if ws == 1 else int(os.environ.get("LOCAL_RANK", "0")))
    pkg_build.build()
    pkg.load()
    fams = [("php", h, pigeonhole(h)) for h in (10, 20, 30, 40, 50)] + \
           [("gt", s, ordering(s)) for s in (10, 20, 30)]
    curves, at_opt = {}, 0
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for fam, size, cnf in fams:
        with pkg.Solver.from_cnf(cnf, restarts=8, lr=LR) as s:
            r = s.solve(10 ** 12, time_limit=args.time_limit, chunk=256)
        t, c = r["trace_time_s"], r["trace_best_cost"]
        keep = [0] + [i for i in range(1, len(c)) if c[i] < c[i - 1]] + [len(c) - 1]
        best = int(c[-1])
        at_opt += best == 1
        curves[f"{fam}{size}"] = {"n": cnf.n, "m": cnf.m, "steps": r["steps"], "seconds": r["elapsed_s"],
                                  "best_cost": best,
                                  "trace": [[round(float(t[i]), 4), int(c[i])] for i in sorted(set(keep))]}
    clk = clocks.stop()
    line = {"metric": "structured families at the optimum (cost 1) within the time limit",
            "value": at_opt, "unit": "instances", "n_gpus": 1, "steps": None, "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": STRUCTURED, "time_limit_s": args.time_limit, "restarts": 8, "lr": LR,
                       "families": "pigeonhole PHP(h) h in {10..50}, ordering GT(s) s in {10, 20, 30}"},
            "curves": curves, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_next_rows(args):
    """Each loss normaliser of the ablation (mean over unsat clauses, sum,
    mean over all clauses) on the default 3-SAT instance with B = 256 for a
    fixed number of steps through msat_solve; per run the best cost, the
    steps to it, and at the end the quick f_j > 0 reading against the exact
    test.  Then a partial MaxSAT instance (planted 3-SAT hard clauses, unit
    soft clauses weighted 1..9, hard weight top = 1 + sum of soft weights)
    solved as one weighted instance: restarts whose best cost is below top
    satisfy every hard clause, and that cost is their soft cost."""
    import torch
    import paper_2402_03640_gb300 as pkg
    from paper_2402_03640_gb300 import build as pkg_build

    ws, rank, _ = dist_env()
    torch.cuda.set_device(0 if ws == 1 else int(os.environ.get("LOCAL_RANK", "0")))
    pkg_build.build()
    pkg.load()
    steps, lr = args.next_steps, 3e-2
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    cnf = WORKLOADS[DENSE_WORKLOAD][0]()
    B = WORKLOADS[DENSE_WORKLOAD][1]
    ablation = {}
    for norm in ("mean_unsat", "sum_unsat", "mean_all"):
        with pkg.Solver.from_cnf(cnf, restarts=B, seed_x=1, lr=lr, loss_norm=norm) as s:
            r = s.solve(steps, chunk=100)
            _, best = s.best()
            bstep = s.best_step()
            hu, dg = s.heuristic_gap()
        b = int(np.argmin(best))
        ablation[norm] = {"steps": int(r["steps"]), "ms_per_step": 1e3 * r["elapsed_s"] / max(1, r["steps"]),
                          "best_cost": int(best.min()), "mean_best_cost": float(best.mean()),
                          "steps_to_best": int(bstep[b]),
                          "quick_reading_unsat_mean": float(hu.mean()),
                          "quick_reading_disagreements_mean": float(dg.mean())}
    n_p, m_hard, m_soft, Bp = 2000, 6000, 2000, 64
    pcnf = random_partial(n_p, m_hard, m_soft, seed=0)
    top = int(pcnf.weights[:m_hard].max())
    with pkg.Solver.from_cnf(pcnf, restarts=Bp, seed_x=1, lr=lr) as s:
        r = s.solve(steps, chunk=100)
        _, best = s.best()
        bstep = s.best_step()
    ok = best < top
    bmin = int(best.min())
    # a cost is top x (hard clauses violated) + soft cost, the soft cost < top
    partial = {"n": n_p, "hard_clauses": m_hard, "soft_clauses": m_soft, "top": top, "restarts": Bp,
               "steps": int(r["steps"]), "ms_per_step": 1e3 * r["elapsed_s"] / max(1, r["steps"]),
               "best_cost": bmin, "best_hard_violated": bmin // top, "best_soft_cost": bmin % top,
               "restarts_with_hard_satisfied": int(ok.sum()),
               "steps_to_best": int(bstep[int(np.argmin(best))])}
    clk = clocks.stop()
    line = {"metric": "best cost after a fixed number of steps (mean-over-unsat loss)",
            "value": ablation["mean_unsat"]["best_cost"], "unit": "weighted unsat clauses", "n_gpus": 1,
            "steps": steps, "warmup": 0, "ms_per_step": ablation["mean_unsat"]["ms_per_step"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": NEXT_ROWS, "instance": DENSE_WORKLOAD, "restarts": B, "lr": lr,
                       "partial_instance": f"planted 3-SAT n={n_p}, {m_hard} hard clauses (seed 0), "
                                           f"{m_soft} unit soft clauses weighted 1..9"},
            "loss_ablation": ablation, "partial_maxsat": partial, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    import torch
    import paper_2402_03640_gb300 as pkg
    from paper_2402_03640_gb300 import build as pkg_build

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    pkg_build.build()
    pkg.load()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    res = serve_compare(pkg, args.serve_requests, args.serve_rate, rank=rank, world=ws)
    clk = clocks.stop()
    value = res["instances_per_s"]
    line = {
        "metric": "instances/s", "value": value, "unit": "instances/s", "n_gpus": ws,
        "steps": res["steps"], "warmup": 1, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": SERVING, "description": res["sample"], "requests": res["requests"],
                   "arrival_rate_per_s": res["arrival_rate_per_s"], "restarts": res["restarts"],
                   "steps_per_request": res["steps"], "l2": "working set of the mix larger than L2"},
        "serving": res, "roofline": None, "cpu_baseline": None, "clocks": clk,
        "e2e": {"value": value, "unit": "instances/s",
                "h2d_bytes_per_step": res["h2d_bytes_per_request"],
                "d2h_bytes_per_step": res["d2h_bytes_per_request"],
                "note": "requests enter as host arrays through msat_submit and leave through msat_wait"},
        "gpu_launches": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# a kernel's sources and those of the data layout it reads (host_cnf.cu
# builds the row order of the stored w f)
KERNEL_SOURCES = {"forward": ("k_step.cu", "msat_internal.cuh", "host_cnf.cu"),
                  "backward": ("k_step.cu", "msat_internal.cuh", "host_cnf.cu"),
                  "dense_eval": ("k_dense.cu", "msat_internal.cuh"),
                  "small_steps": ("k_step.cu", "msat_internal.cuh")}


def kernel_hash(kind="forward"):
    """Hash of a kernel's sources, to tell whether stored ncu traffic is stale."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2402_03640_gb300", "csrc")
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + [SERVING, STRUCTURED, NEXT_ROWS],
                    default=DEFAULT_WORKLOAD)
    ap.add_argument("--next-steps", type=int, default=2000,
                    help="steps of each run of the ablation / partial MaxSAT workload")
    ap.add_argument("--time-limit", type=float, default=1.0,
                    help="seconds per instance of the structured cost-vs-time workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the other configurations and the serving comparison")
    ap.add_argument("--f-mode", choices=("auto", "store", "recompute", "expanded"), default="auto",
                    help="how the variable pass gets f: stored by the clause pass or recomputed")
    ap.add_argument("--shape", default="",
                    help="launch shape FWD_VW:STAGE_VW:LIGHT_ROWS instead of the autotuner's (0 = automatic)")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the serving comparison (0: skip it on the default line)")
    ap.add_argument("--serve-rate", type=float, default=1000.0, help="Poisson arrival rate, requests/s")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == SERVING:
        return run_serving(args)
    if args.workload == STRUCTURED:
        return run_structured(args)
    if args.workload == NEXT_ROWS:
        return run_next_rows(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
