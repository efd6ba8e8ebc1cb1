#!/usr/bin/env python
"""Throughput of sliced circuit tensor-network contraction on GB300.

Default workload: the 36-qubit 6x6 grid circuit of depth 14 with qubits
30..35 left open (64 amplitudes per contraction) and 10 sliced bonds (1024
slices, each contracted and summed in FP64), in the 3xTF32 tensor-core form
with the plain complex64 form and the split-BF16 and FP16-scaled forms timed
beside it, under its stored annealed plan (`--plan local-search` gives the
plan it was annealed from, with the sliced bonds of the workload's seeded
plan; `--plan greedy` the seeded greedy order).  `--workload sliced` runs the 20-qubit 4x5 grid circuit
of depth 12 with 6 sliced bonds for 256 random bitstrings, under its stored
checkpoint plan.  One step = one
full contraction of the workload (every slice for every bitstring) from
device-resident bitstrings to device-resident complex128 amplitudes.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.  Under torchrun each rank
contracts its own 256 bitstrings (weak scaling, no data-path collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from qxgen import circuits as C  # noqa: E402
from qxgen import workloads as W  # noqa: E402

L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
# name -> (C-ABI code, tensor-core products per real MMA, peak ratio to measured BF16)
PRECISIONS = {"c64": (0, 0, 0.0), "3xtf32": (1, 3, 1.1 / 2.25), "bf16x3": (2, 6, 1.0), "fp16": (3, 1, 1.0)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="large", choices=["small", "sliced", "large", "batched", "serving", "sampling"])
    p.add_argument("--sample-batch", type=int, default=1024, help="candidates per contraction when sampling")
    p.add_argument("--samples-per-step", type=int, default=256)
    p.add_argument("--serve-seconds", type=float, default=60.0, help="arrival window of the serving run")
    p.add_argument("--serve-rate", type=float, default=200.0, help="mean requests per second (Poisson)")
    p.add_argument("--serve-max-request-s", type=float, default=1.0,
                   help="largest estimated service time of one request the server admits")
    p.add_argument("--serve-max-backlog-s", type=float, default=0.5,
                   help="estimated work admitted and not yet done beyond which arrivals are shed")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--max-items", type=int, default=0, help="cap on (slice, bitstring) pairs per batch (0 = fill)")
    p.add_argument("--precision", default="3xtf32", choices=list(PRECISIONS),
                   help="contraction form (3xtf32 and bf16x3 meet the 1e-5 tolerance; fp16 is reported)")
    p.add_argument("--executor", default="auto", choices=["auto", "batched", "persistent"])
    p.add_argument("--plan", default="auto",
                   choices=["auto", "level-aware", "greedy", "checkpoint", "local-search", "annealed"],
                   help="auto: the large workload's stored annealed plan (its local-search plan annealed over the "
                        "contraction tree and the choice of the 10 sliced bonds), the sliced workload's stored "
                        "checkpoint plan (its level-aware plan improved by local search: each slice's environment "
                        "contracted once, little work per bitstring); level-aware: the seeded greedy candidate that "
                        "executes the fewest flops per call; greedy: the seeded greedy order of the workload "
                        "definition")
    p.add_argument("--no-forms", action="store_true",
                   help="skip timing the other forms beside (the large workload's split-BF16 and FP16-scaled "
                        "forms; the batched workload's plain complex64 run)")
    p.add_argument("--slices", type=int, default=0,
                   help="contract only slices 0..S-1 per step (a smaller case of the same launches, for profiling; "
                        "the workload name then says so); 0 = all")
    p.add_argument("--workspace-gb", type=float, default=-1.0,
                   help="device workspace of each form (the same for all, so batches match); "
                        "-1: 48 GB for the large workload, else what one call needs up to 60%% of free memory")
    p.add_argument("--no-slice-level", action="store_true",
                   help="compute bitstring-independent intermediates per (slice, bitstring) pair, not per slice")
    p.add_argument("--streams", type=int, default=8,
                   help="streams the batched executor issues independent steps on (1 = in plan order)")
    return p.parse_args()


def workload(name, plan="auto"):
    if name == "sliced" and plan == "level-aware":
        return W.sliced_level_aware()
    if name == "sliced" and plan in ("auto", "checkpoint"):
        return W.sliced_checkpoint()
    if name == "large" and plan in ("auto", "annealed"):
        return W.large_annealed()
    if name == "large" and plan == "local-search":
        return W.large_local_search()
    return {"small": W.small, "sliced": W.sliced, "large": W.large}[name]()


def rank_bits(w, rank):
    if rank == 0:
        return w.bitstrings
    return C.random_bitstrings(w.n_qubits, len(w.bitstrings), w.circuit.seed + 500000 + 7919 * rank)


def config_of(w, extra=None):
    cfg = {"workload": w.name, "n_qubits": w.n_qubits, "depth": w.circuit.depth,
           "grid": f"{w.circuit.rows}x{w.circuit.cols}", "sliced_bonds": len(w.sliced), "slices": w.n_slices,
           "bitstrings_per_gpu": int(len(w.bitstrings)), "open_qubits": w.n_open,
           "amplitudes_per_gpu": int(len(w.bitstrings)) << w.n_open, "peak_entries": 1 << w.peak_rank,
           "plan": w.meta.get("plan", "seeded greedy (order) + tree trimming (slices)"), "precision": None}
    cfg.update(extra or {})
    return cfg


# --------------------------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------------------------------
# CPU oracle leg
# --------------------------------------------------------------------------------------------------
def cpu_oracle_sample(w, n_slices_sample):
    """Time the einsum oracle on 1 bitstring x n_slices_sample slices; returns (amps/s, seconds)."""
    from oracle import einsum as oe
    t0 = time.perf_counter()
    oe.amplitudes(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, w.bitstrings[:1],
                  slices=range(n_slices_sample))
    dt = time.perf_counter() - t0
    amps = (n_slices_sample / w.n_slices) * (1 << w.n_open)
    return amps / dt, dt


def cpu_oracle_timed(w, target_s=10.0):
    """The einsum oracle on successive (bitstring, slice block) samples until target_s of host work;
    returns (amplitudes/s counting a slice block as its share of an amplitude, seconds, samples)."""
    from oracle import einsum as oe
    ns = sample_slices(w)
    blocks = max(w.n_slices // ns, 1)
    t0 = time.perf_counter()
    amps, k = 0.0, 0
    while time.perf_counter() - t0 < target_s:
        b, blk = (k // blocks) % len(w.bitstrings), k % blocks
        oe.amplitudes(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, w.bitstrings[b:b + 1],
                      slices=range(blk * ns, min((blk + 1) * ns, w.n_slices)))
        amps += (min(ns, w.n_slices - blk * ns) / w.n_slices) * (1 << w.n_open)
        k += 1
    dt = time.perf_counter() - t0
    return amps / dt, dt, k


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name on x86; implementer / part ids on Arm)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return None
    for key in ("model name", "Model name"):
        for ln in info.splitlines():
            if ln.startswith(key):
                return ln.split(":", 1)[1].strip()
    impl = sorted({ln.split(":", 1)[1].strip() for ln in info.splitlines() if ln.startswith("CPU implementer")})
    part = sorted({ln.split(":", 1)[1].strip() for ln in info.splitlines() if ln.startswith("CPU part")})
    return f"Arm implementer {','.join(impl)} part {','.join(part)}" if part else None


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def sample_slices(w):
    """Slices of one bitstring the oracle contracts per sample (a few seconds of host work)."""
    return 1 if w.n_slices == 1 else 16 if w.n_slices == 64 else 2


def reference_arm(args, w, rank, world):
    if rank != 0:
        return
    ns = sample_slices(w)
    for _ in range(args.warmup):
        cpu_oracle_sample(w, ns)
    times = []
    for _ in range(args.steps):
        _, dt = cpu_oracle_sample(w, ns)
        times.append(dt)
    amps_per_step = (ns / w.n_slices) * (1 << w.n_open)
    value = amps_per_step * len(times) / sum(times)
    sample = f"1 bitstring x {ns} of {w.n_slices} slices per step (complex128 numpy plan einsum)"
    line = {"impl": "reference", "metric": "amplitudes/s", "value": value, "unit": "amplitudes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": config_of(w, {"sample": sample}),
            "cpu_baseline": {"value": value, "unit": "amplitudes/s", "cores": cpu_threads(), "cpu": cpu_model(),
                             "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------------------
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def traffic_for(kind, workload_name):
    """Per-launch DRAM bytes of a kernel kind on a workload from the committed ncu summary (the mean over
    that kind's launches in one step), if the kernel's source is unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as f:
            d = json.load(f)
        import hashlib
        k = d.get("kernels", {}).get(f"{kind}@{workload_name}")
        if not k:
            return None
        src = os.path.join(ROOT, "paper_2110_09894_gb300", "csrc", k.get("source", ""))
        with open(src, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != k.get("source_sha256"):
                return None
        return k.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        return None


def group_bench(args):
    """All 256 circuits of the uneven batched workload in one captured CUDA graph per step: the light ones
    (intermediates within a CTA's scratch) in the persistent launch, the heavy ones on the batched
    executor, with the autotuned tile family and slice-batch size of each heavy member."""
    import torch
    from paper_2110_09894_gb300 import autotune
    from paper_2110_09894_gb300 import build as qxbuild
    from paper_2110_09894_gb300.batch import UnevenBatch
    qxbuild.build()
    ws = W.batched_members()
    prec = PRECISIONS[args.precision][0]
    t0 = time.perf_counter()
    b, choice, tune_ms = autotune.tuned_uneven(ws, precision=prec)
    tune_s = time.perf_counter() - t0
    b.capture()
    eager = b.amplitudes()
    launches = 3 * (b.group is not None) + sum(c.stats()["launches"] for c in b.heavy_members.values())
    flops = sum(float(c.stats()["flops"]) for c in b.heavy_members.values()) + \
        sum(float(ws[i].flops_per_slice) * ws[i].n_slices * len(ws[i].bitstrings) for i in b.light)
    amps = sum(len(w.bitstrings) << w.n_open for w in ws)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def timed(batch):
        for _ in range(args.warmup):
            batch.replay()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            with torch.cuda.stream(batch.stream):
                flush.fill_(i & 0xFF)
            ev[i][0].record(batch.stream)
            batch.replay()
            ev[i][1].record(batch.stream)
        torch.cuda.synchronize()
        batch.check()
        return [a.elapsed_time(c) for a, c in ev]

    sampler = ClockSampler(0)
    sampler.start()
    ms = timed(b)
    clocks = sampler.stop()
    got = b.amplitudes()
    replay_equal = all(np.array_equal(a, c) for a, c in zip(eager, got))
    # parity of every member against its complex128 state vector (stored by tests/golden/make_batched_golden.py)
    parity = None
    gpath = os.path.join(ROOT, "tests", "golden", "batched_statevector.json")
    if os.path.exists(gpath):
        with open(gpath) as f:
            recs = {r["j"]: r for r in json.load(f)["circuits"]}
        worst_l2 = worst_el = 0.0
        checked = 0
        for w, a in zip(ws, got):
            r = recs.get(w.meta["j"])
            if r is None:
                continue
            ref = (np.array(r["re"]) + 1j * np.array(r["im"])).reshape(a.shape)
            worst_l2 = max(worst_l2, float(np.linalg.norm(a - ref) / np.linalg.norm(ref)))
            worst_el = max(worst_el, float(np.max(np.abs(a - ref)) / np.sqrt(np.mean(np.abs(ref) ** 2))))
            checked += 1
        parity = {"vs": "complex128 state vectors (batched_statevector.json)", "members_checked": checked,
                  "worst_rel_l2": worst_l2, "worst_max_elem_over_rms": worst_el}
    # the same members in plain complex64 (heavy members on the SIMT kernels), same settings
    vs_c64 = None
    if prec != 0 and not args.no_forms:
        b64 = UnevenBatch(ws, precision=0, ctas_per_sm=choice["ctas_per_sm"],
                          settings={int(i): s for i, s in choice["settings"].items()})
        b64.capture()
        ms64 = timed(b64)
        a64 = b64.amplitudes()
        vs_c64 = {"c64_ms_per_step": sum(ms64) / len(ms64), "speedup": sum(ms64) / sum(ms),
                  "worst_rel_diff_to_c64": max(float(np.linalg.norm(x - y) / np.linalg.norm(y))
                                               for x, y in zip(got, a64))}
        b64.close()
    n_light, n_heavy = len(b.light), len(b.heavy)
    line = {"metric": "amplitudes/s", "value": amps * len(ms) / (sum(ms) / 1e3), "unit": "amplitudes/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"c64": "c64", "3xtf32": "tf32x3", "bf16x3": "bf16x3", "fp16": "fp16"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "batched uneven grid circuits (256: n 16..28, depth 8..16, S 0..8, 1..64 "
                                   "bitstrings)", "members": len(ws), "light_persistent": n_light,
                       "heavy_batched": n_heavy, "pairs": int(sum(w.n_slices * len(w.bitstrings) for w in ws)),
                       "amplitudes": int(amps),
                       "executor": "one captured CUDA graph per step: persistent launch (light members, complex64) "
                                   "+ batched launches of the heavy members (" + args.precision + ")",
                       "autotuned": {"ctas_per_sm": choice["ctas_per_sm"], "heavy_settings": choice["settings"]},
                       "autotune_s": tune_s, "l2": "flushed between timed steps"},
            "complex_tflops_executed": flops * len(ms) / (sum(ms) / 1e3) / 1e12, "parity": parity,
            "graph_replay_equals_eager_run": replay_equal, "vs_plain_c64": vs_c64,
            "gpu_launches": int(launches * args.steps), "clocks": clocks}
    b.close()
    print(json.dumps(line), flush=True)


def serving_bench(args):
    """Poisson arrivals on the 32 resident serving circuits, in the chosen form and in plain complex64:
    offered, admitted and completed work, sustained amplitudes/s and latency of completed requests."""
    # one stream per lane and a few dozen lanes: give them hardware queues of their own (a process
    # setting, read when CUDA initialises)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch
    from paper_2110_09894_gb300 import build as qxbuild
    from paper_2110_09894_gb300 import serve
    qxbuild.build()
    ws = [W.serving_circuit(j) for j in range(32)]
    reqs0 = serve.poisson_requests(len(ws), lambda i: ws[i].n_qubits, args.serve_rate, args.serve_seconds, 1024,
                                   5000)
    offered_amps = sum(r.bits.shape[0] for r in reqs0)

    def one_run(precision):
        reqs = [serve.Request(r.rid, r.circuit, r.bits, r.arrival) for r in reqs0]
        srv = serve.Server(ws, precision=precision, max_bits=1024, max_request_s=args.serve_max_request_s,
                           max_backlog_s=args.serve_max_backlog_s, warm=True)
        sampler = ClockSampler(0)
        sampler.start()
        t0 = time.perf_counter()
        done = srv.run(reqs, deadline=args.serve_seconds + 60.0)
        wall = time.perf_counter() - t0
        clocks = sampler.stop()
        summ = serve.latency_summary(done)
        out = {"amplitudes_per_s": summ["amplitudes"] / wall, "wall_s": wall, "completed": summ["completed"],
               "completed_amplitudes": summ["amplitudes"], "admitted": srv.stats["admitted"],
               "rejected_cost": srv.stats["rejected_cost"], "rejected_busy": srv.stats["rejected_busy"],
               "rejected_memory": srv.stats["rejected"] - srv.stats["rejected_cost"] - srv.stats["rejected_busy"],
               "latency_ms": {"p50": summ["p50_ms"], "p99": summ["p99_ms"]},
               "service_over_estimate": {"p50": summ["service_over_estimate_p50"],
                                         "p90": summ["service_over_estimate_p90"]},
               "per_circuit": {str(ci): {"admitted": srv.circuit_stats[ci]["admitted"],
                                         "completed": srv.circuit_stats[ci]["completed"],
                                         "service_over_estimate_p50": float(np.median(
                                             [(r.done - r.started) / max(r.est, 1e-9) for r in done
                                              if r.circuit == ci] or [0.0])),
                                         "est_s_1024_bitstrings": srv.circuits[ci].estimate(1024),
                                         "est_s_1_bitstring": srv.circuits[ci].estimate(1),
                                         "pairs_per_batch": srv.circuits[ci].items}
                               for ci in range(len(ws)) if srv.circuit_stats[ci]["admitted"]},
               "merged_requests": srv.stats["merged_requests"], "chunks": srv.stats["chunks"],
               "lanes": srv.stats["lanes"], "clocks": clocks,
               "servable_circuits": sum(1 for sc in srv.circuits
                                        if sc.servable and sc.estimate(1) <= args.serve_max_request_s)}
        srv.close()
        return out

    main = one_run(PRECISIONS[args.precision][0])
    c64 = one_run(0) if args.precision != "c64" else None
    line = {"metric": "amplitudes/s", "value": main["amplitudes_per_s"], "unit": "amplitudes/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": main["wall_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "serving: 32 resident grid circuits (n 20..40, depth 10..16, peak <= 2^30)",
                       "arrivals": f"Poisson {args.serve_rate}/s for {args.serve_seconds} s, 1..1024 bitstrings",
                       "requests": len(reqs0), "offered_amplitudes": int(offered_amps),
                       "admission": f"memory budget, estimated service <= {args.serve_max_request_s} s, "
                                    f"admitted backlog <= {args.serve_max_backlog_s} s"},
            "latency_ms": main["latency_ms"], "served": main, "plain_c64": c64, "clocks": main["clocks"]}
    print(json.dumps(line), flush=True)


def sampling_bench(args):
    """Output bitstrings of the 20-qubit sliced workload by empirical-supremum rejection sampling (Sec. III-B)."""
    import torch
    from paper_2110_09894_gb300 import build as qxbuild
    from paper_2110_09894_gb300 import qx
    from paper_2110_09894_gb300.sampler import ESupSampler
    qxbuild.build()
    w = W.sliced()
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, args.sample_batch,
                      precision=PRECISIONS[args.precision][0])
    s = ESupSampler(c, seed=1, warmup=2 * args.sample_batch)
    per = args.samples_per_step
    for _ in range(max(args.warmup, 3)):
        s.sample(per)
    it0, con0 = s.iterations, s.contracted
    sampler = ClockSampler(0)
    sampler.start()
    times = []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = s.sample(per)  # synchronous: counts come back to the host every call
        times.append(time.perf_counter() - t0)
        assert x.shape == (per, w.n_qubits)
    clocks = sampler.stop()
    total = sum(times)
    line = {"metric": "samples/s", "value": per * args.steps / total, "unit": "samples/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": "sampling: grid 4x5 depth 12, 6 sliced bonds (64 slices, seeded greedy plan), "
                                   "uniform candidates",
                       "samples_per_step": per, "candidates_per_contraction": s.batch,
                       "warmup_iterations": 2 * args.sample_batch},
            "candidates_per_sample": (s.iterations - it0) / (per * args.steps),
            "amplitudes_per_s": (s.contracted - con0) / total, "bound_m": s.m, "clocks": clocks}
    c.close()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "ours" and args.workload == "batched":
        return group_bench(args)
    if args.impl == "ours" and args.workload == "serving":
        return serving_bench(args)
    if args.impl == "ours" and args.workload == "sampling":
        return sampling_bench(args)
    w = workload(args.workload, args.plan) if args.workload in ("small", "sliced", "large") else W.sliced()
    if args.impl == "reference":
        reference_arm(args, w, rank, world)
        return

    import torch
    from paper_2110_09894_gb300 import build as qxbuild
    if rank == 0 or world == 1:
        qxbuild.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        qxbuild.build()  # no-op once rank 0 built it
    from paper_2110_09894_gb300 import qx
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    bits = rank_bits(w, rank)
    n_bits = len(bits)
    # --slices S: a smaller case of the same launches (slices 0..S-1 of every bitstring, for profiling);
    # a step then yields S / n_slices of each amplitude, counted as that fraction
    s_end = min(args.slices, w.n_slices) if args.slices > 0 else w.n_slices
    amps_per_step = (n_bits << w.n_open) * s_end / w.n_slices
    # host-side build and plan compile, timed apart from the contraction (a host-only handle)
    t0 = time.perf_counter()
    hh = qx.qx_create(-1, precision=PRECISIONS[args.precision][0])
    qx.qx_build_network(hh, w.n_qubits, w.gates, w.open_mask)
    t1 = time.perf_counter()
    qx.qx_set_plan(hh, w.order, w.sliced)
    t2 = time.perf_counter()
    qx.qx_destroy(hh)
    host_ms = {"build_network": 1e3 * (t1 - t0), "set_plan": 1e3 * (t2 - t1)}
    ws_bytes = None
    if args.workspace_gb > 0 or (args.workspace_gb < 0 and args.workload == "large"):
        ws_bytes = int((args.workspace_gb if args.workspace_gb > 0 else 48.0) * 1e9)

    def contractor(precision):
        return qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, n_bits, device=local, stream=stream,
                             max_items=args.max_items, precision=precision, workspace_bytes=ws_bytes,
                             executor={"auto": 0, "batched": 1, "persistent": 2}[args.executor],
                             no_slice_level=int(args.no_slice_level))

    with torch.cuda.stream(stream):
        c = contractor(PRECISIONS[args.precision][0])
        qx.qx_set_streams(c.h, args.streams)
        d_bits = torch.from_numpy(bits).to(dev)
        d_amps = torch.empty((n_bits, 1 << w.n_open, 2), dtype=torch.float64, device=dev)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ws_gb = c.workspace.numel() / 1e9

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        c.contract_device(d_bits, d_amps, s_end=s_end)
    stream.synchronize()
    launches_per_step = c.stats()["launches"]
    flops_exec = c.stats()["flops"]

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)  # evict L2 between timed steps (outside the events)
        ev[i][0].record(stream)
        c.contract_device(d_bits, d_amps, s_end=s_end)
        ev[i][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    my_ms = sum(step_ms)
    t = torch.tensor([my_ms], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    value = amps_per_step * world * args.steps / (max_ms / 1e3)
    ms_per_step = max_ms / args.steps
    # complex flops of the plan as written: 8 M K N per step, for every (slice, bitstring) pair; the
    # executed flops count a step that no output bit touches once per slice (and invariant steps once)
    flops_alg = float(w.flops_per_slice) * w.n_slices * n_bits
    tflops = flops_exec * world * args.steps / (max_ms / 1e3) / 1e12

    # the same steps with the invariant intermediates kept from the first call (qx_set_memo): what a
    # sampler or a server pays per call once the circuit is resident; reported beside, not as value
    qx.qx_set_memo(c.h, 1)
    for _ in range(2):  # computes and keeps them, then captures the graph without those steps
        c.contract_device(d_bits, d_amps, s_end=s_end)
    evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
        evm[i][0].record(stream)
        c.contract_device(d_bits, d_amps, s_end=s_end)
        evm[i][1].record(stream)
    barrier()
    memo_ms = sum(a.elapsed_time(b) for a, b in evm) / args.steps
    memo = {"ms_per_step": memo_ms, "value": amps_per_step / (memo_ms / 1e3),
            "flops_per_step_executed": c.stats()["flops"],
            "what": "invariant intermediates (no sliced bond, no output bit) kept from the first call"}
    qx.qx_set_memo(c.h, 0)

    def as_complex(t):
        x = t.cpu().numpy()
        return x[..., 0] + 1j * x[..., 1]

    def time_form(precision):
        """The same steps in another form (same workspace size, so the same batches): ms per step and
        the device amplitudes of its last step."""
        with torch.cuda.stream(stream):
            cf = contractor(precision)
            qx.qx_set_streams(cf.h, args.streams)
            out = torch.empty_like(d_amps)
        for _ in range(args.warmup):
            cf.contract_device(d_bits, out, s_end=s_end)
        evf = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(i & 0xFF)
            evf[i][0].record(stream)
            cf.contract_device(d_bits, out, s_end=s_end)
            evf[i][1].record(stream)
        barrier()
        qx.qx_device_status(cf.h)
        msf = sum(a.elapsed_time(b) for a, b in evf) / args.steps
        cf.close()
        del cf
        return msf, as_complex(out)

    # the same steps in the plain complex64 form, for the forms' speed-up
    vs_c64 = None
    a_main = as_complex(d_amps)
    a64 = None
    if args.precision != "c64":
        ms64, a64 = time_form(0)
        vs_c64 = {"c64_ms_per_step": ms64, "speedup": ms64 / ms_per_step,
                  "rel_diff_to_c64": float(np.linalg.norm(a_main - a64) / np.linalg.norm(a64))}
    # the other tensor-core forms beside (the large workload runs all three against plain complex64)
    forms = None
    if args.workload == "large" and not args.no_forms:
        forms = {}
        for name in ("3xtf32", "bf16x3", "fp16"):
            if name == args.precision:
                continue
            msf, af = time_form(PRECISIONS[name][0])
            forms[name] = {"ms_per_step": msf, "value": amps_per_step / (msf / 1e3),
                           "speedup_vs_c64": (vs_c64["c64_ms_per_step"] / msf) if vs_c64 else None,
                           "rel_diff_to_c64": float(np.linalg.norm(af - a64) / np.linalg.norm(a64))
                           if a64 is not None else None}

    # per-kernel event timing over K more steps on the same stream
    qx.qx_set_profiling(c.h, True)
    for _ in range(args.steps):
        c.contract_device(d_bits, d_amps, s_end=s_end)
    prof = qx.qx_profile_read(c.h)
    qx.qx_set_profiling(c.h, False)

    # end to end through the public host API: pinned bitstrings in, pinned amplitudes out
    h_bits = torch.from_numpy(bits).pin_memory()
    h_amps = torch.empty((n_bits, 1 << w.n_open, 2), dtype=torch.float64).pin_memory()
    def contract_host():
        if s_end == w.n_slices:
            c.contract_host_ptr(h_bits.data_ptr(), n_bits, h_amps.data_ptr())
        else:
            c.contract_slices_host_ptr(h_bits.data_ptr(), n_bits, 0, s_end, h_amps.data_ptr())

    contract_host()
    barrier()
    lat = []
    t_e2e = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        contract_host()
        lat.append(time.perf_counter() - t0)
    barrier()
    t_e2e = time.perf_counter() - t_e2e
    te = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = amps_per_step * world * args.steps / float(te.item())

    if rank != 0:
        dist.destroy_process_group()
        return

    pk, pk_src = peaks()
    dom = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dom]
    avg_ms = d["ms"] / max(d["launches"], 1)
    # the binding roofline of the dominant kernel: its algorithmic bytes at the measured HBM bandwidth
    # or its operations at the unit's peak, whichever takes longer for the same work
    hbm_peak = pk["hbm_gbs"]
    t_bytes = d["bytes"] / (hbm_peak * 1e9)
    if dom in ("tc_gemm", "tc_direct", "tc_direct_kb"):
        code, products, ratio = PRECISIONS[args.precision]
        peak = pk["bf16_tflops"] * ratio
        ops = d["flops"] * products  # issued real tensor flops
        comp = {"bound": "tensor", "peak": peak, "unit": "TFLOP/s", "issued_products": products,
                "peak_source": f"bf16_tflops ({pk_src}, burst) x {ratio:.3f} nominal {args.precision} ratio"}
    elif dom == "gemm":
        clk = pk.get("sm_max_mhz", 2070.0)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = n_sm * 128 * 2 * clk * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x clock
        ops = d["flops"]
        comp = {"bound": "alu", "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 x {clk:.0f} MHz (max clock)"}
    else:
        ops, comp = 0.0, None
    if comp is not None and ops / (comp["peak"] * 1e12) >= t_bytes:
        achieved = ops / (d["ms"] / 1e3) / 1e12
        roof = dict(comp, achieved=achieved, frac=achieved / comp["peak"],
                    algorithmic_per_launch=ops / max(d["launches"], 1),
                    other_bound={"bound": "hbm", "frac": d["bytes"] / (d["ms"] / 1e3) / 1e9 / hbm_peak})
    else:
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": f"hbm_gbs ({pk_src})", "algorithmic_per_launch": d["bytes"] / max(d["launches"], 1)}
        if comp is not None:
            roof["other_bound"] = {"bound": comp["bound"],
                                   "frac": ops / (d["ms"] / 1e3) / 1e12 / comp["peak"]}
    traffic = traffic_for(dom, w.name)
    roof.update({"kernel": dom, "traffic": traffic, "avg_launch_ms": avg_ms,
                 "share_of_kernel_time": d["ms"] / max(sum(v["ms"] for v in prof.values()), 1e-12)})
    kernels = {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] / args.steps,
                   "tflops": v["flops"] / max(v["ms"], 1e-12) / 1e9, "gbs": v["bytes"] / max(v["ms"], 1e-12) / 1e6}
               for k, v in prof.items()}

    # parity of this launch configuration: the large workload's slices 0..31 against the complex128
    # oracle's partial sum stored by tests/golden/make_large_golden.py (which calls only the oracle)
    parity = None
    if args.workload == "large":
        gname = {"_ls": "large_ls_slices0_31.json", "_sa": "large_sa_slices0_31.json"}.get(w.name[-3:],
                                                                                          "large_slices0_31.json")
        gpath = os.path.join(ROOT, "tests", "golden", gname)
        if os.path.exists(gpath):
            with open(gpath) as f:
                g = json.load(f)
            ref = np.array(g["re"]) + 1j * np.array(g["im"])
            got = c.contract_slices(bits[:1], 0, 32)[0]
            rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
            parity = {"vs": f"complex128 einsum oracle, slices 0..31 ({gname})",
                      "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                      "max_elem_over_rms": float(np.max(np.abs(got - ref)) / rms),
                      "tolerance": {"rel_l2": 1e-5, "max_elem_over_rms": 1e-5 * float(np.sqrt(2 * np.log(2 * ref.size)))}}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        ns = sample_slices(w)
        v, dt, k = cpu_oracle_timed(w)
        cpu = {"value": v, "unit": "amplitudes/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"{k} samples of 1 bitstring x {ns} of {w.n_slices} slices (complex128 numpy plan "
                         f"einsum), {dt:.1f} s of host work",
               "cpu": cpu_model()}
        if w.n_qubits <= 26:
            import oracle
            t0 = time.perf_counter()
            ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, bits)
            cpu["statevector_amplitudes_per_s"] = ref.size / (time.perf_counter() - t0)
            got = d_amps.cpu().numpy()
            got = got[..., 0] + 1j * got[..., 1]
            cpu["rel_err_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    line = {"metric": "amplitudes/s", "value": value, "unit": "amplitudes/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"c64": "c64", "3xtf32": "tf32x3", "bf16x3": "bf16x3", "fp16": "fp16"}[args.precision],
            "data": "synthetic",
            "config": config_of(w, {"workload": w.name + (f"_slices0-{s_end - 1}" if s_end < w.n_slices else ""),
                                    "precision": args.precision + " contraction, FP64 slice sum",
                                    "executor": args.executor, "streams": args.streams,
                                    "bitstring_independent_steps": "per pair" if args.no_slice_level else "per slice",
                                    "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                                    "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write); "
                                          f"workspace {ws_gb:.1f} GB",
                                    "batches_per_step": c.stats()["batches"]}),
            "ms_per_step_median": float(np.median(step_ms)), "host_ms": host_ms,
            "complex_tflops_executed": tflops, "memoised_invariants": memo, "vs_plain_c64": vs_c64,
            "other_forms": forms, "parity": parity, "flops_per_step_algorithmic": flops_alg,
            "flops_per_step_executed": flops_exec,
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))},
            "roofline": roof, "kernels": kernels, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "amplitudes/s", "h2d_bytes_per_step": int(bits.nbytes),
                    "d2h_bytes_per_step": int(h_amps.numel() * 8)},
            "gpu_launches": int(launches_per_step * args.steps), "clocks": clocks, "wall_s_timed": t_wall}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
