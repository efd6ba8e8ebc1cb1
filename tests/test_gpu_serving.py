"""Continuous-batching server: every request's amplitudes match the oracle,
and a request gives the same result alone and in a busy mix (needs a GPU)."""
import numpy as np
import pytest

import oracle
from qxgen import circuits as C
from qxgen.workloads import _workload

from ._util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    from paper_2110_09894_gb300 import build
    build.build()
    from paper_2110_09894_gb300 import serve as mod
    return mod


def _circuits():
    out = []
    for j, (r, c, d, s) in enumerate([(3, 4, 8, 3), (2, 5, 10, 2), (3, 3, 12, 4), (4, 4, 6, 1)]):
        circ = C.random_grid_circuit(r, c, d, 800 + j)
        out.append(_workload(f"srv{j}", circ, np.zeros(circ.n_qubits, np.uint8), s, 800 + j,
                             np.zeros((1, circ.n_qubits), np.uint8)))
    return out


def test_requests_match_oracle_and_alone_equals_mix(serve):
    ws = _circuits()
    reqs = serve.poisson_requests(len(ws), lambda i: ws[i].n_qubits, rate=2000.0, duration=0.05, max_bits=24, seed=5)
    assert len(reqs) > 20
    srv = serve.Server(ws, max_bits=96, chunk_s=1e-6, max_lanes_per_circuit=2)
    done = srv.run(reqs, deadline=120)
    assert len(done) == len(reqs)
    assert srv.stats["chunks"] > srv.stats["batches"]  # long batches ran in several slice chunks
    for r in done:
        w = ws[r.circuit]
        ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, r.bits)
        assert_parity(r.amps, ref)
    summary = serve.latency_summary(done)
    assert summary["completed"] == len(reqs) and summary["p99_ms"] >= summary["p50_ms"] > 0
    srv.close()
    # the same request alone on an idle server
    probe = max(done, key=lambda r: len(r.bits))
    alone = serve.Server(ws, max_bits=96, chunk_s=1e-6)
    one = alone.run([serve.Request(0, probe.circuit, probe.bits, 0.0)], deadline=60)
    assert_parity(one[0].amps, probe.amps)
    alone.close()


def test_memory_admission_rejects_what_cannot_fit(serve):
    ws = _circuits()
    srv = serve.Server(ws, max_bits=8, mem_budget=1 << 10)
    assert not srv.submit(serve.Request(0, 0, np.zeros((1, ws[0].n_qubits), np.uint8), 0.0))
    assert srv.stats["rejected"] == 1


def test_submit_and_poll_requests(serve):
    """qx_submit enqueues without waiting; qx_poll reports each request once, with the same bits as the
    blocking slice-range call; unknown request numbers are an error."""
    import time

    import torch

    from paper_2110_09894_gb300 import qx
    from tests._util import grid_case
    circ, om, order, sliced, bits = grid_case(3, 4, 8, 61, 1, 3, 5)
    st = torch.cuda.Stream()
    c = qx.Contractor(circ.n_qubits, C.gates_to_records(circ), om, order, sliced, 5, stream=st)
    ref = c.contract_slices(bits, 2, 7)
    d_bits = torch.from_numpy(bits).cuda()
    outs, reqs = [], []
    for k in range(3):
        d_amps = torch.empty((5, 2, 2), dtype=torch.float64, device="cuda")
        h_amps = torch.empty((5, 2, 2), dtype=torch.float64).pin_memory()
        reqs.append(qx.qx_submit(c.h, d_bits.data_ptr(), 5, 2, 7, d_amps.data_ptr(), h_amps.data_ptr()))
        outs.append((d_amps, h_amps))
    assert reqs == sorted(reqs) and len(set(reqs)) == 3
    pending, t0 = set(reqs), time.time()
    while pending and time.time() - t0 < 60:
        for r in list(pending):
            if qx.qx_poll(c.h, r):
                pending.discard(r)
    assert not pending
    for d_amps, h_amps in outs:
        got = h_amps.numpy()
        assert np.array_equal(got[..., 0] + 1j * got[..., 1], ref)
        assert np.array_equal(d_amps.cpu().numpy(), got)
    with pytest.raises(qx.QXError):
        qx.qx_poll(c.h, reqs[0])  # reported already
    with pytest.raises(qx.QXError):
        qx.qx_poll(c.h, 10 ** 9)
    qx.qx_device_status(c.h)


def test_parts_of_a_slice_sum_add_like_one_call(serve):
    """qx_submit_part: the FP64 compensated accumulators carry over on the device from part to part, so
    a sum over all slices submitted in parts equals the one-call sum (same per-slice results, same slice
    order); a continuing part that does not follow the open sum is refused."""
    import time

    import torch

    from paper_2110_09894_gb300 import qx
    from tests._util import grid_case
    circ, om, order, sliced, bits = grid_case(3, 4, 8, 62, 1, 4, 6)
    st = torch.cuda.Stream()
    c = qx.Contractor(circ.n_qubits, C.gates_to_records(circ), om, order, sliced, 6, stream=st,
                      executor=qx.EXEC_BATCHED)
    whole = c.contract(bits)
    ref = oracle.sv_amplitudes(circ.n_qubits, C.gates_to_records(circ), om, bits)
    assert_parity(whole, ref)
    d_bits = torch.from_numpy(bits).cuda()
    d_amps = torch.full((6, 2, 2), float("nan"), dtype=torch.float64, device="cuda")
    h_amps = torch.full((6, 2, 2), float("nan"), dtype=torch.float64).pin_memory()
    parts = [(0, 3), (3, 4), (4, 11), (11, 16)]
    reqs = []
    for k, (s0, s1) in enumerate(parts):
        reqs.append(qx.qx_submit_part(c.h, d_bits.data_ptr(), 6, s0, s1, k == 0, k == len(parts) - 1,
                                      d_amps.data_ptr(), h_amps.data_ptr()))
        if k == 1:  # parts before the last write nothing
            st.synchronize()
            assert np.all(np.isnan(h_amps.numpy()))
    t0 = time.time()
    while reqs and time.time() - t0 < 60:
        reqs = [r for r in reqs if not qx.qx_poll(c.h, r)]
    assert not reqs
    got = h_amps.numpy()
    got = got[..., 0] + 1j * got[..., 1]
    assert np.array_equal(got, whole)
    with pytest.raises(qx.QXError) as e:  # no open sum to continue
        qx.qx_submit_part(c.h, d_bits.data_ptr(), 6, 16, 16 + 0, False, True, d_amps.data_ptr())
    r = qx.qx_submit_part(c.h, d_bits.data_ptr(), 6, 0, 5, True, False, d_amps.data_ptr())
    with pytest.raises(qx.QXError) as e:  # skips slices 5..6
        qx.qx_submit_part(c.h, d_bits.data_ptr(), 6, 7, 16, False, True, d_amps.data_ptr())
    assert e.value.code == qx.QX_ESTATE
    qx.qx_device_status(c.h)
    while not qx.qx_poll(c.h, r):
        pass
    c.close()


def _mirror(rows, cols, depth, seed, n_slice):
    """U U^dagger on a rows x cols grid: amp(x) = 1 for x = 0...0 and 0 for every other x, exactly."""
    from qxgen.workloads import make_plan
    u = C.random_grid_circuit(rows, cols, depth, seed)
    m = u.then(u.inverse())
    om = np.zeros(m.n_qubits, np.uint8)
    order, sliced, peak, flops = make_plan(m, om, n_slice, seed + 700000, trials=2)
    from qxgen.workloads import Workload
    return Workload(f"mirror{rows}x{cols}_d{depth}x2", m, om, order, sliced, np.zeros((1, m.n_qubits), np.uint8),
                    peak, flops)


def test_serving_circuits_of_the_workload_and_mirror_pins(serve):
    """Requests on two resident circuits of the serving workload (20 qubits, their stored plans) against
    the state vector, and on 36- and 40-qubit mirror circuits, whose amplitudes are known exactly (1 at
    0...0, 0 elsewhere), in one busy mix: each result also equals the same request served alone."""
    from qxgen import workloads as W
    ws = [W.serving_circuit(7), W.serving_circuit(14), _mirror(6, 6, 4, 9141, 2), _mirror(5, 8, 4, 9144, 3)]
    assert [w.n_qubits for w in ws] == [20, 20, 36, 40]
    reqs = serve.poisson_requests(len(ws), lambda i: ws[i].n_qubits, rate=400.0, duration=0.05, max_bits=16, seed=9)
    for r in reqs:  # every request on a mirror circuit also asks for 0...0
        if ws[r.circuit].n_qubits > 20:
            r.bits[0] = 0
    assert len(reqs) >= 10 and {r.circuit for r in reqs} == {0, 1, 2, 3}
    srv = serve.Server(ws, precision=1, max_bits=64, chunk_s=0.01, max_lanes_per_circuit=2)
    done = srv.run(reqs, deadline=300)
    assert len(done) == len(reqs)
    for r in done:
        w = ws[r.circuit]
        if w.n_qubits == 20:
            ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, r.bits)
        else:
            ref = np.all(r.bits == 0, axis=1).astype(complex)[:, None]
        assert_parity(r.amps, ref, what=w.name)
    srv.close()
    probe = max(done, key=lambda r: len(r.bits) + 100 * (ws[r.circuit].n_qubits == 40))
    alone = serve.Server(ws, precision=1, max_bits=64, chunk_s=0.01)
    one = alone.run([serve.Request(0, probe.circuit, probe.bits, 0.0)], deadline=120)
    assert_parity(one[0].amps, probe.amps)
    alone.close()
