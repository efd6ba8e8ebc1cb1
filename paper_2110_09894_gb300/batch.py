"""Uneven circuits and slice sets contracted together in one captured CUDA graph.

The slices and bitstrings of many circuits are independent units of work
(Sec. IV-A's slice and bitstring levels of parallelism, across circuits).
Members whose intermediates fit one CTA's scratch (at most 2^18 entries per
(slice, bitstring) pair, no tensor-core step) run in the persistent group
launch of the C ABI (qx_group_*: whole contractions per CTA, one FP64 sum);
the others -- large intermediates, tensor-core products -- run on the batched
executor (one launch per step over many pairs, steps at their dependence
level).  Everything is enqueued on one stream and captured as one CUDA graph,
so a step of the whole workload is one graph launch.

Only argument marshalling lives here: every step runs in libqx's kernels.
"""
from __future__ import annotations

from . import qx

LIGHT_MAX_PEAK = 18  # per-pair entries a persistent CTA's scratch holds (2^18 complex64 = 2 MiB)


class UnevenBatch:
    """workloads: objects with n_qubits, gates, open_mask, order, sliced, bitstrings, peak_rank.

    precision applies to the heavy members (the persistent launch runs complex64);
    settings maps a heavy member's index to autotuned Contractor options
    ({"max_items": .., "gemm_min_bits": ..}); mem_budget caps the heavy members'
    workspaces together (bytes, default 60% of the free device memory): each
    keeps its own fixed part, and all share one buffer for their batch regions
    (they run in turn on one stream), as large as the largest whole-call need
    or what the budget leaves."""

    def __init__(self, workloads, device=0, precision=qx.QX_PREC_3XTF32, ctas_per_sm=0, settings=None,
                 mem_budget=None, stream=None):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.dev)
        self.workloads = list(workloads)
        self.light = [i for i, w in enumerate(self.workloads) if w.peak_rank <= LIGHT_MAX_PEAK]
        self.heavy = [i for i, w in enumerate(self.workloads) if w.peak_rank > LIGHT_MAX_PEAK]
        self.precision = precision
        settings = settings or {}
        self.d_bits = [torch.from_numpy(w.bitstrings).to(self.dev) for w in self.workloads]
        torch.cuda.synchronize(self.dev)  # the bitstrings are on the device before the batch's stream reads them
        self.d_amps = [None] * len(self.workloads)
        self.group = None
        with torch.cuda.stream(self.stream):
            if self.light:
                members = [self._contractor(i, qx.QX_PREC_C64, executor=qx.EXEC_GROUP_MEMBER) for i in self.light]
                self.group = qx.Group(members, [self.d_bits[i] for i in self.light], ctas_per_sm)
                for k, i in enumerate(self.light):
                    self.d_amps[i] = self.group.d_amps[k]
                self.light_members = members
            free, _ = torch.cuda.mem_get_info(self.dev)
            budget = int(mem_budget if mem_budget is not None else 0.6 * free)
            # the heavy members run one after another on the batch's stream, so they share one buffer for
            # their per-slice and per-pair regions (qx_bind_workspace_parts); each keeps its own fixed part
            self.heavy_members = {}
            need = {i: self._sizes(i, settings.get(i, {})) for i in self.heavy}
            fixed = sum(f for f, _, _ in need.values())
            lo = max((b1 for _, b1, _ in need.values()), default=0)
            hi = max((bn for _, _, bn in need.values()), default=0)
            batch_bytes = min(hi, budget - fixed)
            if self.heavy and batch_bytes < lo:
                raise MemoryError(f"the heavy members need {fixed + lo} bytes at least; {budget} available")
            self.batch_buffer = (torch.empty(int(batch_bytes), dtype=torch.uint8, device=self.dev)
                                 if self.heavy else None)
            for i in self.heavy:
                s = settings.get(i, {})
                self.heavy_members[i] = self._contractor(i, precision, max_items=s.get("max_items", 0),
                                                         gemm_min_bits=s.get("gemm_min_bits", 0),
                                                         batch_buffer=self.batch_buffer)
                w = self.workloads[i]
                self.d_amps[i] = torch.empty((len(w.bitstrings), 1 << w.n_open, 2), dtype=torch.float64,
                                             device=self.dev)
        torch.cuda.synchronize(self.dev)  # set-up copies and memsets on any stream are done before the first run
        self.graph = None

    def _contractor(self, i, precision, executor=qx.EXEC_BATCHED, max_items=0, gemm_min_bits=0,
                    batch_buffer=None):
        w = self.workloads[i]
        return qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings),
                             device=self.dev.index, precision=precision, max_items=max_items, stream=self.stream,
                             executor=executor, gemm_min_bits=gemm_min_bits, batch_buffer=batch_buffer)

    def _sizes(self, i, s):
        """(fixed part, batch part for one pair, batch part for a whole call) of heavy member i, bytes."""
        w = self.workloads[i]
        h = qx.qx_create(-1, precision=self.precision, max_items=s.get("max_items", 0),
                         gemm_min_bits=s.get("gemm_min_bits", 0))
        try:
            qx.qx_build_network(h, w.n_qubits, w.gates, w.open_mask)
            qx.qx_set_plan(h, w.order, w.sliced)
            nb = len(w.bitstrings)
            pairs = (1 << len(w.sliced)) * nb
            cap = s.get("max_items", 0) or pairs
            fixed, one = qx.qx_workspace_parts(h, nb, 1)
            return fixed, one, qx.qx_workspace_parts(h, nb, min(cap, pairs))[1]
        finally:
            qx.qx_destroy(h)

    def run(self):
        """Enqueue one contraction of every member on the batch's stream (no synchronisation)."""
        with self.torch.cuda.stream(self.stream):
            if self.group is not None:
                self.group.run()
            for i, c in self.heavy_members.items():
                c.contract_device(self.d_bits[i], self.d_amps[i])

    def capture(self):
        """Run once eagerly (uploads, stream and event creation), then capture one run as a CUDA graph."""
        torch = self.torch
        self.run()
        self.stream.synchronize()
        self.check()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self.run()
        return self.graph

    def replay(self):
        with self.torch.cuda.stream(self.stream):
            self.graph.replay()

    def check(self):
        """Device status of every heavy member (a bounded wait that expired raises QXError)."""
        for c in self.heavy_members.values():
            qx.qx_device_status(c.h)

    def amplitudes(self):
        out = []
        for a in self.d_amps:
            h = a.cpu().numpy()
            out.append(h[..., 0] + 1j * h[..., 1])
        return out

    def close(self):
        if self.group is not None:
            self.group.close()
            self.group = None
        for c in list(self.heavy_members.values()) + list(getattr(self, "light_members", [])):
            c.close()
        self.heavy_members = {}
