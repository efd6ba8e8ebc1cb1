"""Shared helpers for the tests: tolerances and small workload builders."""
import json
import os

import numpy as np

from qxgen import circuits as C
from qxgen.workloads import make_plan

# Plain complex64 path: relative l2 error over a request's amplitudes <= 1e-5
# against the complex128 oracle.  Each step rounds every product once in FP32
# (unit roundoff 6e-8) and there are a few hundred steps, so the expected error
# is ~1e-6; 1e-5 is the stated acceptance level.
TOL_C64 = 1e-5


# Element-wise: the largest error of any single amplitude, relative to the rms magnitude of the
# oracle's amplitudes in the same request (a relative error per amplitude is unstable for random-
# circuit amplitudes near zero, Porter-Thomas).  FP32 rounding gives every amplitude of a request an
# error of about the same scale sigma, independently, and the largest of N such errors stays below
# sigma * sqrt(2 ln 2N) (Gaussian tail), so an l2 error at the 1e-5 tolerance allows a largest
# element error of TOL_C64 * sqrt(2 ln 2N) times the rms amplitude (1.2e-5 for one amplitude, 3.1e-5
# for 64, 3.5e-5 for 256).  An error confined to a few amplitudes, which the l2 norm over the request
# could hide, fails it: one amplitude carrying the whole l2 budget is sqrt(N) * 1e-5 times the rms.
def tol_elem(n):
    return TOL_C64 * float(np.sqrt(2.0 * np.log(2.0 * max(int(n), 1))))


def rel_l2(a, ref):
    a = np.asarray(a).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    return float(np.linalg.norm(a - ref) / max(np.linalg.norm(ref), 1e-300))


def max_elem(a, ref):
    """max_i |a_i - ref_i| / rms_i |ref_i|."""
    a = np.asarray(a).reshape(-1)
    ref = np.asarray(ref).reshape(-1)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2)) if ref.size else 0.0
    return float(np.max(np.abs(a - ref)) / max(rms, 1e-300)) if ref.size else 0.0


def _log(kind, l2, el):
    path = os.environ.get("QX_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "kind": kind,
                                "rel_l2": l2, "max_elem": el}) + "\n")


def assert_parity(a, ref, tol=TOL_C64, what=""):
    """Both parity bounds of a request: relative l2 over its amplitudes and the element-wise bound."""
    l2, el = rel_l2(a, ref), max_elem(a, ref)
    te = tol / TOL_C64 * tol_elem(np.asarray(ref).size)
    _log(what, l2, el)
    assert l2 <= tol, f"{what} relative l2 error {l2:.3e} > {tol:.0e}"
    assert el <= te, f"{what} largest element error {el:.3e} x rms > {te:.2e}"


def grid_case(rows, cols, depth, seed, n_open=0, n_slice=0, n_bits=8, trials=0):
    circ = C.random_grid_circuit(rows, cols, depth, seed)
    n = circ.n_qubits
    om = np.zeros(n, np.uint8)
    if n_open:
        om[n - n_open:] = 1
    order, sliced, peak, flops = make_plan(circ, om, n_slice, seed + 700000, trials)
    bits = C.random_bitstrings(n, n_bits, seed + 500000)
    return circ, om, order, sliced, bits


def cancelling_slices_case():
    """A 2-qubit network whose four slice results are X, 1, -X, -1 (X = 2^60, slice order), all exact
    in FP32: their exact sum is 0, a plain running FP64 sum in slice order gives -1 (X + 1 rounds to X),
    a compensated one gives 0.  Gates need not be unitary for the method (explicit matrices).

    Bonds: 0, 1 inputs; 2 (qubit 0) and 3 (qubit 1) between the two layers of gates (sliced);
    4, 5 the final wires.  Slice s sets bond 2 to bit 0 of s and bond 3 to bit 1.
    """
    from qxgen.plan import greedy_order, network_legs
    X = 2.0 ** 60
    circ = C.Circuit(2)
    circ.append([0], [[X, 0], [1, 0]])
    circ.append([1], [[1, 0], [-1, 0]])
    circ.append([0], [[1, 1], [0, 0]])
    circ.append([1], [[1, 1], [0, 0]])
    om = np.zeros(2, np.uint8)
    legs, _, _ = network_legs(2, [g.qubits for g in circ.gates], om)
    order = greedy_order(legs)
    bits = np.zeros((1, 2), np.uint8)
    return circ, om, order, [2, 3], bits
