"""Tensor-core precision forms (tcgen05 3xTF32 and 3-way split BF16) against
the complex128 oracle, through the C ABI (needs a GPU).

Both compensated forms must meet the same relative l2 tolerance as the plain
complex64 path; the large workload's long reductions (K up to 2^15) are the
stress case for FP32 accumulation in TMEM.
"""
import json
import os

import numpy as np
import pytest

import oracle
from qxgen import workloads as W

from ._util import assert_parity, grid_case, rel_l2

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
FORMS = [1, 2]  # QX_PREC_3XTF32, QX_PREC_SPLIT_BF16


@pytest.fixture(scope="module")
def qx():
    from paper_2110_09894_gb300 import build
    build.build()
    from paper_2110_09894_gb300 import qx as mod
    return mod


def _tc_launches(qx, c, run):
    qx.qx_set_profiling(c.h, True)
    out = run()
    prof = qx.qx_profile_read(c.h)
    qx.qx_set_profiling(c.h, False)
    return out, prof["tc_gemm"]["launches"] + prof["tc_direct"]["launches"] + prof["tc_direct_kb"]["launches"]


@pytest.mark.parametrize("precision", FORMS)
def test_forms_on_sliced_workload(qx, precision):
    w = W.sliced()
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings), precision=precision)
    got, n_tc = _tc_launches(qx, c, lambda: c.contract(w.bitstrings))
    assert n_tc > 0, "no step ran on the tensor cores"
    assert_parity(got, ref)
    c.close()


@pytest.mark.parametrize("precision", FORMS)
def test_forms_with_open_legs_and_ragged_batches(qx, precision):
    circ, om, order, sliced, bits = grid_case(4, 5, 10, 64, n_open=3, n_slice=4, n_bits=5)
    from qxgen import circuits as C
    recs = C.gates_to_records(circ)
    ref = oracle.sv_amplitudes(circ.n_qubits, recs, om, bits)
    c = qx.Contractor(circ.n_qubits, recs, om, order, sliced, len(bits), precision=precision, max_items=7)
    got = c.contract(bits)
    assert_parity(got, ref)


LARGE = {"greedy": ("large", "large_slices0_31.json"),
         "local-search": ("large_local_search", "large_ls_slices0_31.json"),
         "annealed": ("large_annealed", "large_sa_slices0_31.json")}


@pytest.mark.parametrize("plan", list(LARGE))
@pytest.mark.parametrize("precision", FORMS)
def test_forms_on_large_workload_32_slices(qx, precision, plan):
    fn, name = LARGE[plan]
    w = getattr(W, fn)()
    with open(os.path.join(HERE, "golden", name)) as f:
        g = json.load(f)
    ref = np.array(g["re"]) + 1j * np.array(g["im"])
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 1, precision=precision)
    got, n_tc = _tc_launches(qx, c, lambda: c.contract_slices(w.bitstrings, 0, 32)[0])
    assert n_tc > 0
    assert_parity(got, ref)


def test_fp16_scaled_form_runs_on_tensor_cores_and_reports_its_error(qx, capsys):
    """FP16 with per-tensor power-of-two scales: its error is reported, not held to 1e-5."""
    w = W.sliced()
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings),
                      precision=qx.QX_PREC_FP16_SCALED)
    got, n_tc = _tc_launches(qx, c, lambda: c.contract(w.bitstrings))
    err = rel_l2(got, ref)
    with capsys.disabled():
        print(f"\nFP16-scaled relative l2 error on the 4x5 depth-12 workload: {err:.3e}")
    assert n_tc > 0
    assert err < 2e-2  # ~2^-11 per element over a few tensor-core steps; a sanity bound only
