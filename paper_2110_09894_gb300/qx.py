"""Python binding of libqx (ctypes, argument marshalling only).

Each function has the name of the C entry point it calls (include/qx.h);
``Contractor`` bundles them with a torch-allocated workspace.  Every step of
the contraction runs in the library's CUDA kernels; if the library is not
built, loading fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

QX_OK, QX_EINVAL, QX_ENOMEM, QX_ECUDA, QX_ETIMEOUT, QX_ESTATE = 0, -1, -2, -3, -4, -5
QX_PREC_C64, QX_PREC_3XTF32, QX_PREC_SPLIT_BF16, QX_PREC_FP16_SCALED = 0, 1, 2, 3
_NAMES = {QX_EINVAL: "QX_EINVAL", QX_ENOMEM: "QX_ENOMEM", QX_ECUDA: "QX_ECUDA", QX_ETIMEOUT: "QX_ETIMEOUT",
          QX_ESTATE: "QX_ESTATE"}

# Entry points declared in include/qx.h (checked by the CPU test-suite).
EXPORTS = ("qx_create", "qx_destroy", "qx_last_error", "qx_set_options", "qx_build_network", "qx_network_info",
           "qx_set_plan", "qx_workspace_size", "qx_bind_workspace", "qx_contract", "qx_contract_device",
           "qx_contract_slices", "qx_contract_slices_device", "qx_last_stats", "qx_set_profiling",
           "qx_profile_read", "qx_contract_device_static", "qx_device_status", "qx_group_create",
           "qx_group_scratch_size", "qx_group_bind", "qx_group_run", "qx_group_last_error", "qx_group_destroy",
           "qx_set_graphs", "qx_set_streams", "qx_describe_plan", "qx_submit", "qx_poll", "qx_esup_accept",
           "qx_esup_sample", "qx_set_memo", "qx_submit_part", "qx_workspace_parts",
           "qx_bind_workspace_parts")
QX_STATIC_SCRATCH_BYTES = 64 << 20
KERNEL_KINDS = ("permute", "small", "gemm", "sum", "tc_prep", "tc_gemm", "persist", "wave", "small_flat", "tc_direct",
                "tc_direct_kb")


class QXError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_items", ctypes.c_int32), ("gemm_min_bits", ctypes.c_int32),
                ("executor", ctypes.c_int32), ("timeout_cycles", ctypes.c_int64), ("no_slice_level", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


_lib = None


def library_path():
    return _build.LIB


def load(path=None):
    """Load libqx.so; raises if it has not been built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise ImportError(f"libqx is not built ({p} missing); run paper_2110_09894_gb300.build.build()")
    lib = ctypes.CDLL(p)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "qx_create": ([ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(Options)], ctypes.c_int),
        "qx_destroy": ([vp], None),
        "qx_last_error": ([vp], ctypes.c_char_p),
        "qx_set_options": ([vp, ctypes.POINTER(Options)], ctypes.c_int),
        "qx_build_network": ([vp, i32, vp, i64, vp], ctypes.c_int),
        "qx_network_info": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "qx_set_plan": ([vp, vp, i64, vp, i32, ctypes.POINTER(i64)], ctypes.c_int),
        "qx_workspace_size": ([vp, i64, i64, ctypes.POINTER(i64)], ctypes.c_int),
        "qx_bind_workspace": ([vp, vp, i64, i64], ctypes.c_int),
        "qx_workspace_parts": ([vp, i64, i64, ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "qx_bind_workspace_parts": ([vp, vp, i64, vp, i64, i64], ctypes.c_int),
        "qx_contract": ([vp, vp, i64, vp], ctypes.c_int),
        "qx_contract_device": ([vp, vp, i64, vp], ctypes.c_int),
        "qx_contract_slices": ([vp, vp, i64, i64, i64, vp], ctypes.c_int),
        "qx_contract_slices_device": ([vp, vp, i64, i64, i64, vp], ctypes.c_int),
        "qx_last_stats": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), ctypes.POINTER(i64)],
                          ctypes.c_int),
        "qx_set_profiling": ([vp, ctypes.c_int], ctypes.c_int),
        "qx_device_status": ([vp], ctypes.c_int),
        "qx_set_graphs": ([vp, ctypes.c_int], ctypes.c_int),
        "qx_set_memo": ([vp, ctypes.c_int], ctypes.c_int),
        "qx_set_streams": ([vp, i32], ctypes.c_int),
        "qx_submit": ([vp, vp, i64, i64, i64, vp, vp, ctypes.POINTER(i64)], ctypes.c_int),
        "qx_poll": ([vp, i64, ctypes.POINTER(i32)], ctypes.c_int),
        "qx_submit_part": ([vp, vp, i64, i64, i64, i32, i32, vp, vp, ctypes.POINTER(i64)], ctypes.c_int),
        "qx_describe_plan": ([vp, ctypes.c_char_p, i64, ctypes.POINTER(i64)], ctypes.c_int),
        "qx_group_create": ([ctypes.POINTER(vp), ctypes.POINTER(vp), i32, ctypes.POINTER(vp), ctypes.POINTER(i64),
                             ctypes.POINTER(vp), i32], ctypes.c_int),
        "qx_group_scratch_size": ([vp, ctypes.POINTER(i64)], ctypes.c_int),
        "qx_group_bind": ([vp, vp, i64], ctypes.c_int),
        "qx_group_run": ([vp], ctypes.c_int),
        "qx_group_last_error": ([vp], ctypes.c_char_p),
        "qx_group_destroy": ([vp], None),
        "qx_contract_device_static": ([vp, vp, i64, vp], ctypes.c_int),
        "qx_esup_accept": ([vp, vp, vp, i64, i32, i64, i64, ctypes.POINTER(ctypes.c_double), vp,
                            ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "qx_esup_sample": ([vp, vp, vp, i64, i64, i64, ctypes.POINTER(ctypes.c_double), vp, vp,
                            ctypes.POINTER(i64), ctypes.POINTER(i64)], ctypes.c_int),
        "qx_profile_read": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = lib
    return lib


def _check(h, rc):
    if rc != QX_OK:
        msg = load().qx_last_error(h)
        raise QXError(rc, msg.decode() if msg else "")


# --- thin wrappers with the C names --------------------------------------------------------------

EXEC_AUTO, EXEC_BATCHED, EXEC_PERSISTENT, EXEC_GROUP_MEMBER = 0, 1, 2, 3


def qx_create(device=0, stream=0, precision=QX_PREC_C64, max_items=0, gemm_min_bits=0, executor=EXEC_AUTO,
              no_slice_level=0, timeout_cycles=0):
    h = ctypes.c_void_p()
    opt = Options(precision, max_items, gemm_min_bits, executor, int(timeout_cycles), int(no_slice_level), 0)
    rc = load().qx_create(ctypes.byref(h), int(device), ctypes.c_void_p(int(stream)), ctypes.byref(opt))
    if rc != QX_OK:
        raise QXError(rc, "qx_create failed (device, options)")
    return h


def qx_destroy(h):
    load().qx_destroy(h)


def qx_last_error(h):
    return load().qx_last_error(h).decode()


def qx_set_options(h, precision=QX_PREC_C64, max_items=0, gemm_min_bits=0, executor=EXEC_AUTO, no_slice_level=0,
                   timeout_cycles=0):
    opt = Options(precision, max_items, gemm_min_bits, executor, int(timeout_cycles), int(no_slice_level), 0)
    _check(h, load().qx_set_options(h, ctypes.byref(opt)))


def qx_build_network(h, n_qubits, gate_records, open_mask=None):
    recs = np.ascontiguousarray(gate_records)
    if recs.dtype.itemsize != 272:
        raise ValueError("gate records must be 272-byte qx_gate structs")
    om = None if open_mask is None else np.ascontiguousarray(np.asarray(open_mask, dtype=np.uint8))
    _check(h, load().qx_build_network(h, int(n_qubits), recs.ctypes.data if len(recs) else None, len(recs),
                                      None if om is None else om.ctypes.data))


def qx_network_info(h):
    nt, nb = ctypes.c_int64(), ctypes.c_int64()
    _check(h, load().qx_network_info(h, ctypes.byref(nt), ctypes.byref(nb)))
    return nt.value, nb.value


def qx_set_plan(h, order, sliced):
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int64).reshape(-1, 2))
    s = np.ascontiguousarray(np.asarray(sliced, dtype=np.int64).reshape(-1))
    peak = ctypes.c_int64()
    _check(h, load().qx_set_plan(h, o.ctypes.data if len(o) else None, len(o), s.ctypes.data if len(s) else None,
                                 len(s), ctypes.byref(peak)))
    return peak.value


def qx_workspace_size(h, max_bits, items):
    b = ctypes.c_int64()
    _check(h, load().qx_workspace_size(h, int(max_bits), int(items), ctypes.byref(b)))
    return b.value


def qx_workspace_parts(h, max_bits, items):
    """(fixed bytes, batch bytes) of a two-part workspace."""
    f, b = ctypes.c_int64(), ctypes.c_int64()
    _check(h, load().qx_workspace_parts(h, int(max_bits), int(items), ctypes.byref(f), ctypes.byref(b)))
    return f.value, b.value


def qx_bind_workspace_parts(h, d_fixed, fixed_bytes, d_batch, batch_bytes, max_bits):
    _check(h, load().qx_bind_workspace_parts(h, ctypes.c_void_p(int(d_fixed)), int(fixed_bytes),
                                             ctypes.c_void_p(int(d_batch)), int(batch_bytes), int(max_bits)))


def qx_bind_workspace(h, dptr, nbytes, max_bits):
    _check(h, load().qx_bind_workspace(h, ctypes.c_void_p(int(dptr) if dptr else 0), int(nbytes), int(max_bits)))


def qx_contract(h, bitstrings, n_qubits, n_open):
    bits = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint8).reshape(-1, n_qubits))
    out = np.empty((len(bits), 1 << n_open), dtype=np.complex128)
    _check(h, load().qx_contract(h, bits.ctypes.data, len(bits), out.ctypes.data))
    return out


def qx_contract_slices(h, bitstrings, n_qubits, n_open, s_begin, s_end):
    bits = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint8).reshape(-1, n_qubits))
    out = np.empty((len(bits), 1 << n_open), dtype=np.complex128)
    _check(h, load().qx_contract_slices(h, bits.ctypes.data, len(bits), int(s_begin), int(s_end), out.ctypes.data))
    return out


def qx_contract_slices_device(h, d_bits_ptr, n_bits, s_begin, s_end, d_amps_ptr):
    _check(h, load().qx_contract_slices_device(h, ctypes.c_void_p(int(d_bits_ptr)), int(n_bits), int(s_begin),
                                               int(s_end), ctypes.c_void_p(int(d_amps_ptr))))


def qx_contract_device(h, d_bits_ptr, n_bits, d_amps_ptr):
    _check(h, load().qx_contract_device(h, ctypes.c_void_p(int(d_bits_ptr)), int(n_bits),
                                        ctypes.c_void_p(int(d_amps_ptr))))


def qx_contract_device_static(h, d_bits_ptr, n_bits, d_amps_ptr):
    """Contract with the library's built-in scratch array: nothing is allocated."""
    _check(h, load().qx_contract_device_static(h, ctypes.c_void_p(int(d_bits_ptr)), int(n_bits),
                                               ctypes.c_void_p(int(d_amps_ptr))))


def qx_esup_accept(h, d_amps_ptr, d_uniforms_ptr, n_cand, n_qubits, n_warmup, max_out, m, d_accepted_ptr):
    """Rejection tests of the empirical-supremum sampler over given amplitudes.

    Returns (accepted count, iterations consumed, bound M after them)."""
    mm, na, nc = ctypes.c_double(m), ctypes.c_int64(), ctypes.c_int64()
    _check(h, load().qx_esup_accept(h, ctypes.c_void_p(int(d_amps_ptr)), ctypes.c_void_p(int(d_uniforms_ptr)),
                                    int(n_cand), int(n_qubits), int(n_warmup), int(max_out), ctypes.byref(mm),
                                    ctypes.c_void_p(int(d_accepted_ptr)), ctypes.byref(na), ctypes.byref(nc)))
    return na.value, nc.value, mm.value


def qx_esup_sample(h, d_cand_ptr, d_uniforms_ptr, n_cand, n_warmup, max_out, m, d_amps_ptr, d_accepted_ptr):
    """Contract the candidates, then run the sampler's tests over them.

    Returns (accepted count, iterations consumed, bound M after them)."""
    mm, na, nc = ctypes.c_double(m), ctypes.c_int64(), ctypes.c_int64()
    _check(h, load().qx_esup_sample(h, ctypes.c_void_p(int(d_cand_ptr)), ctypes.c_void_p(int(d_uniforms_ptr)),
                                    int(n_cand), int(n_warmup), int(max_out), ctypes.byref(mm),
                                    ctypes.c_void_p(int(d_amps_ptr)), ctypes.c_void_p(int(d_accepted_ptr)),
                                    ctypes.byref(na), ctypes.byref(nc)))
    return na.value, nc.value, mm.value


def qx_describe_plan(h):
    need = ctypes.c_int64()
    _check(h, load().qx_describe_plan(h, None, 0, ctypes.byref(need)))
    buf = ctypes.create_string_buffer(need.value)
    _check(h, load().qx_describe_plan(h, buf, need.value, None))
    return buf.value.decode()


def qx_set_graphs(h, enable):
    _check(h, load().qx_set_graphs(h, 1 if enable else 0))


def qx_set_memo(h, enable):
    """Keep the invariant intermediates in the workspace across calls (enable) or recompute them."""
    _check(h, load().qx_set_memo(h, int(enable)))


def qx_submit(h, d_bits_ptr, n_bits, s_begin, s_end, d_amps_ptr, h_amps_ptr=None):
    """Enqueue a slice-range contraction (device buffers; optional pinned host copy); returns the request."""
    req = ctypes.c_int64()
    _check(h, load().qx_submit(h, ctypes.c_void_p(int(d_bits_ptr)), int(n_bits), int(s_begin), int(s_end),
                               ctypes.c_void_p(int(d_amps_ptr)),
                               ctypes.c_void_p(int(h_amps_ptr)) if h_amps_ptr else None, ctypes.byref(req)))
    return req.value


def qx_submit_part(h, d_bits_ptr, n_bits, s_begin, s_end, first, last, d_amps_ptr, h_amps_ptr=None):
    """Enqueue one part of a slice sum (the accumulators carry over between parts); returns the request."""
    req = ctypes.c_int64()
    _check(h, load().qx_submit_part(h, ctypes.c_void_p(int(d_bits_ptr)), int(n_bits), int(s_begin), int(s_end),
                                    int(bool(first)), int(bool(last)), ctypes.c_void_p(int(d_amps_ptr)),
                                    ctypes.c_void_p(int(h_amps_ptr)) if h_amps_ptr else None, ctypes.byref(req)))
    return req.value


def qx_poll(h, req):
    """True once request `req` has finished (reported once), False while it runs."""
    done = ctypes.c_int32()
    _check(h, load().qx_poll(h, int(req), ctypes.byref(done)))
    return bool(done.value)


def qx_set_streams(h, n_streams):
    _check(h, load().qx_set_streams(h, int(n_streams)))


def qx_device_status(h):
    _check(h, load().qx_device_status(h))


def qx_last_stats(h):
    f, l, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check(h, load().qx_last_stats(h, ctypes.byref(f), ctypes.byref(l), ctypes.byref(b)))
    return {"flops": f.value, "launches": l.value, "batches": b.value}


def qx_set_profiling(h, enable):
    _check(h, load().qx_set_profiling(h, 1 if enable else 0))


def qx_profile_read(h):
    """{kind: {ms, launches, flops, bytes}} for every kernel kind."""
    out = {}
    for k, name in enumerate(KERNEL_KINDS):
        ms, n, f, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(h, load().qx_profile_read(h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(f), ctypes.byref(b)))
        out[name] = {"ms": ms.value, "launches": n.value, "flops": f.value, "bytes": b.value}
    return out


# --- convenience ----------------------------------------------------------------------------------

class Contractor:
    """A network + plan resident on one GPU with a torch-allocated workspace."""

    def __init__(self, n_qubits, gate_records, open_mask, order, sliced, max_bits, device=0,
                 precision=QX_PREC_C64, max_items=0, workspace_bytes=None, stream=None, executor=EXEC_AUTO,
                 no_slice_level=0, gemm_min_bits=0, timeout_cycles=0, batch_buffer=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.n_qubits = int(n_qubits)
        self.n_open = 0 if open_mask is None else int(np.sum(np.asarray(open_mask) != 0))
        self.h = qx_create(device, self.stream.cuda_stream, precision, max_items, gemm_min_bits, executor,
                           no_slice_level, timeout_cycles)
        qx_build_network(self.h, n_qubits, gate_records, open_mask)
        self.peak_entries = qx_set_plan(self.h, order, sliced)
        self.n_slices = 1 << len(np.asarray(sliced).reshape(-1))
        self.max_bits = int(max_bits)
        if batch_buffer is not None:
            # two-part workspace: own fixed part, batch regions in a caller-shared torch uint8 buffer
            fixed, _ = qx_workspace_parts(self.h, max_bits, 1)
            self.workspace = torch.empty(int(fixed), dtype=torch.uint8, device=self.device)
            self.batch_buffer = batch_buffer
            qx_bind_workspace_parts(self.h, self.workspace.data_ptr(), int(fixed), batch_buffer.data_ptr(),
                                    batch_buffer.numel(), max_bits)
            return
        if workspace_bytes is None and executor == EXEC_GROUP_MEMBER:
            workspace_bytes = qx_workspace_size(self.h, max_bits, 1)  # pair scratch comes from the group
        if workspace_bytes is None:
            want = qx_workspace_size(self.h, max_bits, self.n_slices * max_bits)
            free, _ = torch.cuda.mem_get_info(self.device)
            workspace_bytes = min(want, int(free * 0.6))
            workspace_bytes = max(workspace_bytes, qx_workspace_size(self.h, max_bits, 1))
        self.workspace = torch.empty(int(workspace_bytes), dtype=torch.uint8, device=self.device)
        qx_bind_workspace(self.h, self.workspace.data_ptr(), workspace_bytes, max_bits)

    def contract(self, bitstrings):
        """Host bitstrings in, host complex128 amplitudes out (copies inside)."""
        return qx_contract(self.h, bitstrings, self.n_qubits, self.n_open)

    def contract_host_ptr(self, bits_ptr, n_bits, amps_ptr):
        """qx_contract on raw host pointers (e.g. pinned buffers); synchronises."""
        _check(self.h, load().qx_contract(self.h, ctypes.c_void_p(int(bits_ptr)), int(n_bits),
                                          ctypes.c_void_p(int(amps_ptr))))

    def contract_slices_host_ptr(self, bits_ptr, n_bits, s_begin, s_end, amps_ptr):
        """qx_contract_slices on raw host pointers (e.g. pinned buffers); synchronises."""
        _check(self.h, load().qx_contract_slices(self.h, ctypes.c_void_p(int(bits_ptr)), int(n_bits), int(s_begin),
                                                 int(s_end), ctypes.c_void_p(int(amps_ptr))))

    def contract_slices(self, bitstrings, s_begin, s_end):
        """Partial sum over slices [s_begin, s_end) (host in, host out)."""
        return qx_contract_slices(self.h, bitstrings, self.n_qubits, self.n_open, s_begin, s_end)

    def contract_device(self, d_bits, d_amps=None, s_begin=0, s_end=None):
        """Device uint8 [n_bits, n_qubits] in, device float64 [n_bits, 2^open, 2] out (enqueued only)."""
        torch = self.torch
        n_bits = d_bits.shape[0]
        if d_amps is None:
            d_amps = torch.empty((n_bits, 1 << self.n_open, 2), dtype=torch.float64, device=self.device)
        s_end = self.n_slices if s_end is None else s_end
        qx_contract_slices_device(self.h, d_bits.data_ptr(), n_bits, s_begin, s_end, d_amps.data_ptr())
        return d_amps

    def stats(self):
        return qx_last_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            qx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _gcheck(g, rc):
    if rc != QX_OK:
        msg = load().qx_group_last_error(g)
        raise QXError(rc, msg.decode() if msg else "")


class Group:
    """Many Contractors (created with executor=EXEC_GROUP_MEMBER) run by one persistent launch.

    `run()` only enqueues work on member 0's stream; `capture()` records it in a
    CUDA graph and `replay()` launches the graph.
    """

    def __init__(self, members, d_bits, ctas_per_sm=0):
        import torch
        self.torch = torch
        self.members = list(members)
        self.d_bits = list(d_bits)
        dev = self.members[0].device
        self.d_amps = [torch.empty((b.shape[0], 1 << m.n_open, 2), dtype=torch.float64, device=dev)
                       for m, b in zip(self.members, self.d_bits)]
        n = len(self.members)
        hs = (ctypes.c_void_p * n)(*[m.h.value for m in self.members])
        bits = (ctypes.c_void_p * n)(*[b.data_ptr() for b in self.d_bits])
        nb = (ctypes.c_int64 * n)(*[b.shape[0] for b in self.d_bits])
        amps = (ctypes.c_void_p * n)(*[a.data_ptr() for a in self.d_amps])
        g = ctypes.c_void_p()
        rc = load().qx_group_create(ctypes.byref(g), hs, n, bits, nb, amps, int(ctas_per_sm))
        self.g = g
        _gcheck(g, rc)
        size = ctypes.c_int64()
        _gcheck(g, load().qx_group_scratch_size(g, ctypes.byref(size)))
        self.scratch = torch.empty(max(size.value, 256), dtype=torch.uint8, device=dev)
        _gcheck(g, load().qx_group_bind(g, self.scratch.data_ptr(), self.scratch.numel()))
        self.graph = None

    def run(self):
        _gcheck(self.g, load().qx_group_run(self.g))

    def capture(self):
        torch = self.torch
        stream = self.members[0].stream
        self.run()  # warm-up outside the capture
        stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=stream):
            self.run()
        return self.graph

    def replay(self):
        # a CUDA graph replays into the current stream: make it the members' stream
        with self.torch.cuda.stream(self.members[0].stream):
            self.graph.replay()

    def amplitudes(self):
        out = []
        for a in self.d_amps:
            h = a.cpu().numpy()
            out.append(h[..., 0] + 1j * h[..., 1])
        return out

    def close(self):
        if getattr(self, "g", None):
            load().qx_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
