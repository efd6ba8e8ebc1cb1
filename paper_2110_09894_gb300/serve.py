"""Continuous-batching amplitude server over resident networks.

Requests (circuit id, bitstrings) arrive over time.  Every circuit keeps its
network, plan and tensors resident in device memory; the server admits work
while other work is on the GPU:

* requests for the same circuit that wait together are merged into one
  contraction (their bitstrings concatenated: the slice-batched executor then
  runs all their (slice, bitstring) pairs in the same launches);
* a merged batch runs in slice chunks of about chunk_s estimated seconds, so
  a long request never holds the GPU for long and new arrivals start between
  chunks; the chunks are parts of one sum in the library (``qx_submit_part``):
  the lane's FP64 compensated accumulators carry from chunk to chunk on the
  device, so a chunked request gets the same sum, in the same slice order, as
  one call over all slices (Eq. 2);
* each circuit owns a few execution lanes (a library handle with its own
  workspace, CUDA stream and request buffers, allocated once); lanes are
  created on demand (or at start, `warm`) while the device memory budget
  allows (admission by memory) and reused afterwards; a lane keeps its
  circuit's invariant intermediates across requests (qx_set_memo);
* each chunk is one asynchronous request of the library (the contraction of
  its slices, and for the last chunk the copy of the amplitudes to pinned
  host memory, on the lane's stream); completion is polled with ``qx_poll``;
  latency runs from a request's arrival to the host seeing its amplitudes;
* a request is rejected at arrival if its circuit cannot get a lane within
  the memory budget (admission by memory), if its estimated service time
  exceeds max_request_s, or if the estimated work already admitted and not
  yet done plus its own exceeds max_backlog_s (load shedding: under an
  offered load beyond the GPU, admitted requests keep a bounded latency
  instead of every request waiting in an unbounded queue).  Service times
  are estimated from the library's compiled launch list of the circuit's
  plan (cost.launch_list_time), linear in the number of bitstrings.

The scheduling runs on the host in Python (it only marshals work); every
contraction step runs in the library's kernels.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import qx
from .cost import launch_list_time


@dataclass
class Request:
    rid: int
    circuit: int
    bits: np.ndarray            # [n, n_qubits] uint8
    arrival: float              # seconds (server clock)
    done: float = -1.0
    amps: np.ndarray | None = None
    est: float = 0.0            # estimated service seconds (set at admission)
    started: float = -1.0       # when its batch started on a lane (server clock)


@dataclass
class _Batch:
    reqs: list
    n: int                      # bitstrings of the merged requests (rows of the lane's buffers in use)
    chunks: list                # [(b0, b1, s0, s1, first, last)] still to run: bitstrings [b0, b1) of
                                # the batch, slices [s0, s1), whether the part starts / ends its sum
    req: int = 0                # library request number of the chunk in flight
    inflight: tuple = None


class _Lane:
    def __init__(self, circ, dev, precision, max_bits, executor):
        import torch
        self.stream = torch.cuda.Stream(dev)
        self.c = qx.Contractor(circ.n_qubits, circ.gates, circ.open_mask, circ.order, circ.sliced, max_bits,
                               device=dev.index or 0, precision=precision, stream=self.stream, executor=executor,
                               workspace_bytes=circ.lane_bytes)
        # every request of the lane's circuit reads the same invariant intermediates: keep them
        qx.qx_set_memo(self.c.h, 1)
        # lanes already overlap on their own streams: a lane issues its launches in plan order on one
        qx.qx_set_streams(self.c.h, 1)
        # request buffers for up to max_bits bitstrings, allocated once (pinned host memory for the copies)
        n_o = 1 << circ.n_open
        self.bits_host = torch.empty((max_bits, circ.n_qubits), dtype=torch.uint8).pin_memory()
        self.bits_dev = torch.empty((max_bits, circ.n_qubits), dtype=torch.uint8, device=dev)
        self.amps_dev = torch.empty((max_bits, n_o, 2), dtype=torch.float64, device=dev)
        self.amps_host = torch.empty((max_bits, n_o, 2), dtype=torch.float64).pin_memory()
        self.batch = None


@dataclass
class ServedCircuit:
    n_qubits: int
    gates: np.ndarray
    open_mask: np.ndarray
    order: list
    sliced: list
    flops_per_slice: float
    n_open: int = 0
    n_slices: int = 1
    lane_bytes: int = 0
    servable: bool = True
    est_a: float = 0.0          # estimated seconds of one batch of b bitstrings: est_a + est_b * b
    est_b: float = 0.0
    items: int = 1              # (slice, bitstring) pairs per batch in a lane's workspace
    slice_ops: int = 0          # launches per batch of the per-slice and the per-pair steps
    pair_ops: int = 0

    def piece(self, n_bits):
        """Bitstrings per piece of a request: a lane runs a request as pieces of at most one batch of
        its workspace, each a sum of its own, so that one library call enqueues a bounded amount of
        work."""
        return max(1, min(n_bits, self.items))

    def estimate(self, n_bits, launch_s=1e-5):
        """Estimated seconds of a request: per piece its work (whole slices with all the piece's
        bitstrings per batch, the launches of every extra batch counted) and its fixed part."""
        total, left = 0.0, n_bits
        while left > 0:
            pn = self.piece(left)
            per = max(1, self.items // pn)
            extra = (-(-self.n_slices // per) - 1) * (self.slice_ops + self.pair_ops)
            total += self.est_a + self.est_b * pn + extra * launch_s
            left -= pn
        return total
    lanes: list = field(default_factory=list)
    queue: collections.deque = field(default_factory=collections.deque)


class Server:
    def __init__(self, circuits, device=0, precision=qx.QX_PREC_C64, max_bits=1024, mem_budget=None,
                 chunk_s=0.05, max_lanes_per_circuit=2, items_per_lane=4096, max_request_s=float("inf"),
                 max_backlog_s=float("inf"), warm=False):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.precision = precision
        self.max_bits = max_bits
        self.chunk_s = chunk_s
        self.max_lanes = max_lanes_per_circuit
        self.max_request_s = max_request_s
        self.max_backlog_s = max_backlog_s
        self.backlog = 0.0
        free, _ = torch.cuda.mem_get_info(self.dev)
        self.budget = int(mem_budget if mem_budget is not None else free * 0.7)
        self.committed = 0
        self.circuits = []
        for w in circuits:
            sc = ServedCircuit(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, float(w.flops_per_slice),
                               n_open=int(np.sum(w.open_mask)), n_slices=1 << len(w.sliced))
            h = qx.qx_create(-1, precision=precision)
            qx.qx_build_network(h, w.n_qubits, w.gates, w.open_mask)
            qx.qx_set_plan(h, w.order, w.sliced)
            # pairs per batch: as many as a lane's share of the budget holds (every circuit can hold a
            # lane at once)
            one = qx.qx_workspace_size(h, max_bits, 1)
            per_pair = max(qx.qx_workspace_size(h, max_bits, 2) - one, 1)
            fit = (self.budget // (2 * max(len(circuits), 4)) - one) // per_pair
            items = int(max(1, min(items_per_lane, sc.n_slices * max_bits, fit)))
            sc.items = items
            sc.lane_bytes = qx.qx_workspace_size(h, max_bits, items)
            sc.servable = sc.lane_bytes <= self.budget
            desc = qx.qx_describe_plan(h)
            lv = [ln.split()[3] for ln in desc.splitlines()]
            sc.slice_ops, sc.pair_ops = lv.count("slice"), lv.count("pair")
            t1 = launch_list_time(desc, sc.n_slices, 1)
            sc.est_b = max((launch_list_time(desc, sc.n_slices, 256) - t1) / 255.0, 0.0)
            sc.est_a = t1 - sc.est_b
            qx.qx_destroy(h)
            self.circuits.append(sc)
        self.clock0 = time.perf_counter()
        self.done = []
        self.stats = collections.Counter()
        self.circuit_stats = [collections.Counter() for _ in self.circuits]
        if warm:
            self._warm()

    def _warm(self):
        """Resident circuits: one lane per circuit that a request can be admitted for (within the memory
        budget, one bitstring within max_request_s), its tensors uploaded and its invariant intermediates
        computed by one contraction of one bitstring, before the first request arrives."""
        torch = self.torch
        for ci, sc in enumerate(self.circuits):
            if not sc.servable or sc.estimate(1) > self.max_request_s:
                continue
            lane = self._free_lane(ci)
            if lane is None:
                continue
            with torch.cuda.stream(lane.stream):
                d_bits = torch.zeros((1, sc.n_qubits), dtype=torch.uint8, device=self.dev)
                lane.c.contract_device(d_bits)
            lane.stream.synchronize()
            qx.qx_device_status(lane.c.h)
            self.stats["warm_lanes"] += 1

    def now(self):
        return time.perf_counter() - self.clock0

    # -- admission ----------------------------------------------------------------------------------
    def _can_lane(self, sc):
        return bool(sc.lanes) or self.committed + sc.lane_bytes <= self.budget

    def _free_lane(self, ci):
        sc = self.circuits[ci]
        for lane in sc.lanes:
            if lane.batch is None:
                return lane
        if len(sc.lanes) < self.max_lanes and self.committed + sc.lane_bytes <= self.budget:
            lane = _Lane(sc, self.dev, self.precision, self.max_bits, qx.EXEC_BATCHED)
            sc.lanes.append(lane)
            self.committed += sc.lane_bytes
            self.stats["lanes"] += 1
            return lane
        return None

    def submit(self, req: Request):
        sc = self.circuits[req.circuit]
        if not sc.servable or len(req.bits) > self.max_bits or not self._can_lane(sc):
            # needs more device memory than the budget holds for it now, or too many bitstrings
            self.stats["rejected"] += 1
            return False
        req.est = sc.estimate(len(req.bits))
        if req.est > self.max_request_s:
            self.stats["rejected"] += 1  # more work than the server accepts for one request
            self.stats["rejected_cost"] += 1
            return False
        if self.backlog + req.est > self.max_backlog_s:
            self.stats["rejected"] += 1  # the GPU is already committed beyond the backlog bound
            self.stats["rejected_busy"] += 1
            return False
        self.backlog += req.est
        self.stats["admitted"] += 1
        self.circuit_stats[req.circuit]["admitted"] += 1
        sc.queue.append(req)
        return True

    def _start(self, ci, lane):
        torch = self.torch
        sc = self.circuits[ci]
        reqs, n = [], 0
        while sc.queue and n + len(sc.queue[0].bits) <= self.max_bits:
            r = sc.queue.popleft()
            reqs.append(r)
            n += len(r.bits)
        if not reqs:
            return False
        bh = lane.bits_host.numpy()
        k = 0
        for r in reqs:
            bh[k:k + len(r.bits)] = r.bits
            k += len(r.bits)
        with torch.cuda.stream(lane.stream):
            lane.bits_dev[:n].copy_(lane.bits_host[:n], non_blocking=True)
        # pieces of at most one batch of the lane's workspace worth of bitstrings (separate sums), each in
        # slice chunks of about chunk_s estimated seconds (parts of one sum): every library call then
        # enqueues a bounded amount of work, so the loop keeps admitting and starting other requests
        piece = sc.piece(n)
        chunks = []
        for b0 in range(0, n, piece):
            b1 = min(n, b0 + piece)
            n_chunks = int(max(1, min(sc.n_slices, sc.estimate(b1 - b0) // self.chunk_s)))
            step = -(-sc.n_slices // n_chunks)
            ranges = [(s0, min(s0 + step, sc.n_slices)) for s0 in range(0, sc.n_slices, step)]
            chunks += [(b0, b1, s0, s1, k == 0, k == len(ranges) - 1) for k, (s0, s1) in enumerate(ranges)]
        lane.batch = _Batch(reqs, n, chunks)
        t_start = self.now()
        for r in reqs:
            r.started = t_start
        self.stats["batches"] += 1
        self.stats["merged_requests"] += len(reqs) - 1
        self._launch_chunk(lane)
        return True

    def _launch_chunk(self, lane):
        b = lane.batch
        b0, b1, s0, s1, first, last = b.chunks.pop(0)
        nq, row = lane.bits_dev.shape[1], lane.amps_dev[0].numel() * 8
        b.req = qx.qx_submit_part(lane.c.h, lane.bits_dev.data_ptr() + b0 * nq, b1 - b0, s0, s1, first, last,
                                  lane.amps_dev.data_ptr() + b0 * row,
                                  (lane.amps_host.data_ptr() + b0 * row) if last else None)
        b.inflight = (b0, b1, s0, s1)
        self.stats["chunks"] += 1

    def _finish_chunk(self, lane):
        b = lane.batch
        if b.chunks:
            self._launch_chunk(lane)
            return
        tot = lane.amps_host.numpy()[:b.n]
        amps = tot[..., 0] + 1j * tot[..., 1]
        t_done = self.now()
        k = 0
        for r in b.reqs:
            r.amps = amps[k:k + len(r.bits)].copy()
            k += len(r.bits)
            r.done = t_done
            self.backlog -= r.est
            self.circuit_stats[r.circuit]["completed"] += 1
            self.done.append(r)
        lane.batch = None

    # -- the loop -----------------------------------------------------------------------------------
    def poll(self):
        """Retire finished chunks, start queued work on free lanes; returns True if anything is in flight."""
        busy = False
        for sc in self.circuits:
            for lane in sc.lanes:
                if lane.batch is not None and qx.qx_poll(lane.c.h, lane.batch.req):
                    self._finish_chunk(lane)
        for ci, sc in enumerate(self.circuits):
            while sc.queue:
                lane = self._free_lane(ci)
                if lane is None or not self._start(ci, lane):
                    break
        for sc in self.circuits:
            busy = busy or any(l.batch is not None for l in sc.lanes) or bool(sc.queue)
        return busy

    def run(self, requests, deadline=None, idle_sleep=2e-4):
        """Feed `requests` (sorted by arrival) in real time; returns when all are done or at `deadline`."""
        i = 0
        self.clock0 = time.perf_counter()
        while True:
            t = self.now()
            while i < len(requests) and requests[i].arrival <= t:
                self.submit(requests[i])
                i += 1
            busy = self.poll()
            if i >= len(requests) and not busy:
                break
            if deadline is not None and t > deadline:
                break
            if not busy:
                time.sleep(idle_sleep)
        return self.done

    def close(self):
        self.torch.cuda.synchronize(self.dev)
        for sc in self.circuits:
            for lane in sc.lanes:
                lane.c.close()
            sc.lanes.clear()


def poisson_requests(n_circuits, n_qubits_of, rate, duration, max_bits, seed):
    """Seeded Poisson arrivals: exponential gaps of mean 1/rate, circuits and sizes uniform."""
    from qxgen.circuits import SplitMix64, random_bitstrings
    rng = SplitMix64(seed)
    reqs, t, rid = [], 0.0, 0
    while True:
        t += -np.log(1.0 - rng.uniform()) / rate
        if t > duration:
            break
        ci = rng.randint(n_circuits)
        nb = 1 + rng.randint(max_bits)
        bits = random_bitstrings(n_qubits_of(ci), nb, seed * 7919 + rid)
        reqs.append(Request(rid, ci, bits, t))
        rid += 1
    return reqs


def latency_summary(done):
    lat = np.array([r.done - r.arrival for r in done]) if done else np.zeros(0)
    amps = sum(r.amps.size for r in done)
    # service time of a batch against the estimate the admission used (merged requests share a batch)
    svc = np.array([(r.done - r.started) / max(r.est, 1e-9) for r in done if r.started >= 0]) if done else np.zeros(0)
    return {"completed": len(done), "amplitudes": int(amps),
            "service_over_estimate_p50": float(np.percentile(svc, 50)) if len(svc) else None,
            "service_over_estimate_p90": float(np.percentile(svc, 90)) if len(svc) else None,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None}
