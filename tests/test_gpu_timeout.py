"""Bounded device waits in the tensor-core kernels (needs a GPU).

Every mbarrier wait of the tcgen05 kernels gives up after the handle's
timeout_cycles; the kernel then records QX_ETIMEOUT, waits for the copies and
MMAs it issued itself (with a fixed bound of its own, not the caller's limit),
frees TMEM and returns, so the context stays usable.  A limit of one cycle is
shorter than any pipeline stage: the first wait that does not succeed at once
gives up.  Nothing faults or hangs; the next call with the default limit must
give the oracle's amplitudes.
"""
import numpy as np
import pytest

import oracle
from qxgen import workloads as W

from ._util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qx():
    from paper_2110_09894_gb300 import build
    build.build()
    from paper_2110_09894_gb300 import qx as mod
    return mod


# QX_PREC_3XTF32 runs the per-pair steps of this plan on the direct kernel (k_gemm_tc2),
# QX_PREC_SPLIT_BF16 runs every tensor-core step on the prep-based kernel (k_gemm_tc)
@pytest.mark.parametrize("precision", [1, 2])
def test_expired_wait_reports_timeout_then_next_call_is_exact(qx, precision):
    w = W.sliced()
    bits = w.bitstrings[:16]
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, bits)
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(bits), precision=precision)
    qx.qx_set_options(c.h, precision=precision, timeout_cycles=1)
    qx.qx_set_profiling(c.h, True)
    with pytest.raises(qx.QXError) as e:
        c.contract(bits)
    assert e.value.code == qx.QX_ETIMEOUT
    prof = qx.qx_profile_read(c.h)
    kinds = ("tc_direct", "tc_direct_kb") if precision == 1 else ("tc_gemm",)
    assert sum(prof[k]["launches"] for k in kinds) > 0
    qx.qx_set_profiling(c.h, False)
    # the default limit again: the same handle, workspace and context give the exact result
    qx.qx_set_options(c.h, precision=precision)
    for _ in range(2):  # eager, then graph capture + replay
        assert_parity(c.contract(bits), ref)
    qx.qx_device_status(c.h)
    c.close()


def test_timeout_of_enqueue_only_call_shows_in_device_status(qx):
    import torch
    w = W.sliced()
    bits = w.bitstrings[:8]
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, bits)
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(bits), precision=1)
    d_bits = torch.from_numpy(np.ascontiguousarray(bits)).cuda()
    qx.qx_set_options(c.h, precision=1, timeout_cycles=1)
    c.contract_device(d_bits)  # enqueues only
    with pytest.raises(qx.QXError) as e:
        qx.qx_device_status(c.h)
    assert e.value.code == qx.QX_ETIMEOUT
    qx.qx_set_options(c.h, precision=1)
    out = c.contract_device(d_bits)
    qx.qx_device_status(c.h)
    a = out.cpu().numpy()
    assert_parity(a[..., 0] + 1j * a[..., 1], ref)
    c.close()
