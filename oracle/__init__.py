"""Independent complex128 CPU oracle for circuit tensor-network amplitudes.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this package; the library never does, and it
shares no code with the CUDA path.

* ``statevector`` / ``sv_amplitudes``: state-vector evolution in C (Sec. II).
* ``einsum.amplitudes``: plan-following pairwise contraction with slicing
  (Sec. II closing of outputs, Sec. III-A order and Eq. 2 slicing), numpy.
* ``sampler.esup_run``: empirical-supremum rejection sampling of output
  bitstrings from candidate amplitudes (Sec. III-B), plain Python.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import einsum  # noqa: F401
from . import sampler  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libqxoracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the C part of the oracle (gcc, OpenMP) into oracle/_build."""
    src = os.path.join(_HERE, "statevector.c")
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # -fcx-limited-range: complex products as (ac - bd, ad + bc) without the library call that only
    # matters for infinities and NaNs (the oracle's values are finite)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fcx-limited-range", "-fPIC", "-shared", src,
                           "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.qxo_sv_evolve.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
            lib.qxo_sv_evolve.restype = ctypes.c_int
            lib.qxo_sv_read.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p]
            lib.qxo_sv_read.restype = ctypes.c_int
            _lib = lib
    return _lib


def statevector(n_qubits, gate_records):
    """complex128 state C|0...0> (qubit 0 = most significant index bit)."""
    lib = _load()
    recs = np.ascontiguousarray(gate_records)
    psi = np.empty(1 << n_qubits, dtype=np.complex128)
    rc = lib.qxo_sv_evolve(n_qubits, recs.ctypes.data, len(recs), psi.ctypes.data)
    if rc != 0:
        raise ValueError("malformed circuit")
    return psi


def sv_read(n_qubits, psi, open_mask, bitstrings):
    lib = _load()
    bits = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint8).reshape(-1, n_qubits))
    om = np.ascontiguousarray(np.zeros(n_qubits, np.uint8) if open_mask is None else np.asarray(open_mask, np.uint8))
    n_open = int(np.sum(om != 0))
    out = np.empty((len(bits), 1 << n_open), dtype=np.complex128)
    rc = lib.qxo_sv_read(n_qubits, np.ascontiguousarray(psi).ctypes.data, om.ctypes.data, bits.ctypes.data,
                         len(bits), out.ctypes.data)
    if rc != 0:
        raise ValueError("bitstrings must be 0/1")
    return out


def sv_amplitudes(n_qubits, gate_records, open_mask, bitstrings):
    """Amplitudes read from the evolved state, laid out like the C-ABI output."""
    return sv_read(n_qubits, statevector(n_qubits, gate_records), open_mask, bitstrings)
