"""Shared helpers for the tests: tolerances and small workload builders."""
import numpy as np

from qxgen import circuits as C
from qxgen.workloads import make_plan

# Plain complex64 path: relative l2 error over a request's amplitudes <= 1e-5
# against the complex128 oracle.  Each step rounds every product once in FP32
# (unit roundoff 6e-8) and there are a few hundred steps, so the expected error
# is ~1e-6; 1e-5 is the stated acceptance level.
TOL_C64 = 1e-5


def rel_l2(a, ref):
    a = np.asarray(a).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    return float(np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-300))


def grid_case(rows, cols, depth, seed, n_open=0, n_slice=0, n_bits=8, trials=0):
    circ = C.random_grid_circuit(rows, cols, depth, seed)
    n = circ.n_qubits
    om = np.zeros(n, np.uint8)
    if n_open:
        om[n - n_open:] = 1
    order, sliced, peak, flops = make_plan(circ, om, n_slice, seed + 700000, trials)
    bits = C.random_bitstrings(n, n_bits, seed + 500000)
    return circ, om, order, sliced, bits
