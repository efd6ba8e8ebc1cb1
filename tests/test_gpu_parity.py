"""CUDA path vs the complex128 oracle, through the C ABI (needs a GPU).

Element-by-element comparisons on seeded inputs at sizes the oracle finishes
in seconds (several tiles, ragged batches), plus the full-size workloads in
the launch configuration the benchmark uses, and closed-form cases.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import einsum as oe
from qxgen import circuits as C
from qxgen import workloads as W

from ._util import assert_parity, grid_case, rel_l2

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def qx():
    from paper_2110_09894_gb300 import build
    build.build()
    from paper_2110_09894_gb300 import qx as mod
    return mod


def _contractor(qx, circ, om, order, sliced, max_bits, **kw):
    return qx.Contractor(circ.n_qubits, C.gates_to_records(circ), om, order, sliced, max_bits, **kw)


def test_small_workload_vs_statevector(qx):
    w = W.small()
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings))
    got = c.contract(w.bitstrings)
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
    assert_parity(got, ref)
    assert c.stats()["launches"] > 0


def test_sliced_workload_vs_statevector_and_unsliced(qx):
    w = W.sliced()
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings))
    got = c.contract(w.bitstrings)
    assert_parity(got, ref)
    # per-bitstring relative error too (amplitudes of a 20-qubit random circuit are ~1e-3)
    per = np.abs(got - ref).reshape(-1) / np.sqrt(np.mean(np.abs(ref) ** 2))
    assert per.max() < 1e-4
    c.close()
    u = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, [], len(w.bitstrings))
    unsliced = u.contract(w.bitstrings)
    assert_parity(unsliced, ref)


@pytest.mark.parametrize("rows,cols,depth,n_open,n_slice,n_bits", [
    (3, 3, 8, 3, 2, 5), (2, 5, 10, 0, 4, 33), (3, 4, 6, 2, 3, 1), (4, 4, 8, 4, 5, 7)])
def test_grid_cases_vs_statevector(qx, rows, cols, depth, n_open, n_slice, n_bits):
    circ, om, order, sliced, bits = grid_case(rows, cols, depth, 31 + depth, n_open, n_slice, n_bits)
    c = _contractor(qx, circ, om, order, sliced, n_bits)
    got = c.contract(bits)
    ref = oracle.sv_amplitudes(circ.n_qubits, C.gates_to_records(circ), om, bits)
    assert got.shape == ref.shape
    assert_parity(got, ref)


@pytest.mark.parametrize("max_items", [1, 3, 64, 0])
def test_batch_size_does_not_change_the_result(qx, max_items):
    circ, om, order, sliced, bits = grid_case(3, 4, 8, 77, 1, 4, 6)
    base = _contractor(qx, circ, om, order, sliced, 6, max_items=1, executor=qx.EXEC_BATCHED).contract(bits)
    got = _contractor(qx, circ, om, order, sliced, 6, max_items=max_items, executor=qx.EXEC_BATCHED).contract(bits)
    assert np.array_equal(got, base)  # same per-pair kernels, same slice order in the FP64 sum


def test_ghz_closed_form(qx):
    n = 12
    circ = C.ghz_circuit(n)
    om = np.zeros(n, np.uint8)
    from qxgen.workloads import make_plan
    order, sliced, _, _ = make_plan(circ, om, 3, 5)
    bits = np.array([[0] * n, [1] * n, [0, 1] * (n // 2)], np.uint8)
    got = _contractor(qx, circ, om, order, sliced, 3).contract(bits)[:, 0]
    s = 1 / math.sqrt(2)
    assert np.allclose(got, [s, s, 0], atol=1e-6)


def test_product_state_closed_form(qx):
    n = 10
    circ = C.product_circuit(n, 4, seed=3)
    v = [np.eye(2, dtype=np.complex128) for _ in range(n)]
    for g in circ.gates:
        v[g.qubits[0]] = g.matrix @ v[g.qubits[0]]
    bits = C.random_bitstrings(n, 9, 4)
    want = np.array([np.prod([v[q][x[q], 0] for q in range(n)]) for x in bits])
    from qxgen.workloads import make_plan
    om = np.zeros(n, np.uint8)
    order, sliced, _, _ = make_plan(circ, om, 0, 1)
    got = _contractor(qx, circ, om, order, sliced, 9).contract(bits)[:, 0]
    assert_parity(got, want)


def test_all_open_no_slices_gives_the_state(qx):
    # every tensor is then independent of slices and bitstrings (prologue only)
    circ, om, order, sliced, bits = grid_case(2, 4, 6, 12, n_open=8, n_slice=0, n_bits=2)
    got = _contractor(qx, circ, om, order, sliced, 2).contract(bits)
    psi = oracle.statevector(8, C.gates_to_records(circ))
    assert_parity(got[0], psi)
    assert np.array_equal(got[0], got[1])
    assert abs(np.sum(np.abs(got[0]) ** 2) - 1) < 1e-5


def test_trivial_networks(qx):
    # one qubit, no gates: <x|0>
    circ = C.Circuit(1)
    c = _contractor(qx, circ, np.zeros(1, np.uint8), [(0, 1)], [], 2)
    got = c.contract(np.array([[0], [1]], np.uint8))[:, 0]
    assert np.allclose(got, [1, 0])


def test_mirror_circuit_36_qubits(qx):
    u = C.random_grid_circuit(6, 6, 3, 55)
    circ = u.then(u.inverse())
    from qxgen.workloads import make_plan
    om = np.zeros(36, np.uint8)
    order, sliced, _, _ = make_plan(circ, om, 3, 9)
    bits = np.concatenate([np.zeros((1, 36), np.uint8), C.random_bitstrings(36, 3, 8)])
    got = _contractor(qx, circ, om, order, sliced, 4).contract(bits)[:, 0]
    assert abs(got[0] - 1) < 1e-5
    assert np.all(np.abs(got[1:]) < 1e-5)


def test_slice_ranges_add_up_and_match_oracle(qx):
    circ, om, order, sliced, bits = grid_case(3, 4, 8, 91, 2, 4, 3)
    c = _contractor(qx, circ, om, order, sliced, 3)
    full = c.contract(bits)
    parts = c.contract_slices(bits, 0, 5) + c.contract_slices(bits, 5, 16)
    assert rel_l2(parts, full) < 1e-12
    ref = oe.amplitudes(circ.n_qubits, C.gates_to_records(circ), om, order, sliced, bits, slices=range(5, 16))
    assert_parity(c.contract_slices(bits, 5, 16), ref)


def test_device_path_matches_host_path(qx):
    import torch
    circ, om, order, sliced, bits = grid_case(3, 4, 8, 5, 1, 3, 9)
    c = _contractor(qx, circ, om, order, sliced, 9)
    host = c.contract(bits)
    d_bits = torch.from_numpy(bits).cuda()
    d_amps = c.contract_device(d_bits)
    torch.cuda.synchronize()
    dev = d_amps.cpu().numpy()
    assert np.array_equal(dev[..., 0] + 1j * dev[..., 1], host)


def test_errors_through_the_abi(qx):
    circ, om, order, sliced, bits = grid_case(2, 3, 4, 5, 0, 1, 2)
    c = _contractor(qx, circ, om, order, sliced, 2)
    bad = bits.copy()
    bad[0, 0] = 2
    with pytest.raises(qx.QXError) as e:
        c.contract(bad)
    assert e.value.code == qx.QX_EINVAL
    with pytest.raises(qx.QXError) as e:
        c.contract(np.zeros((3, 6), np.uint8))
    assert e.value.code == qx.QX_ENOMEM
    with pytest.raises(qx.QXError) as e:
        c.contract_slices(bits, 1, 1)
    assert e.value.code == qx.QX_EINVAL
    h = qx.qx_create(0)
    qx.qx_build_network(h, circ.n_qubits, C.gates_to_records(circ), om)
    with pytest.raises(qx.QXError) as e:
        qx.qx_contract(h, bits, circ.n_qubits, 0)
    assert e.value.code == qx.QX_ESTATE
    qx.qx_destroy(h)


def _golden_large(name="large_slices0_31.json"):
    p = os.path.join(HERE, "golden", name)
    with open(p) as f:
        g = json.load(f)
    return g, np.array(g["re"]) + 1j * np.array(g["im"])


LARGE_PLANS = {"greedy": ("large", "large_slices0_31.json"),
               "local-search": ("large_local_search", "large_ls_slices0_31.json"),
               "annealed": ("large_annealed", "large_sa_slices0_31.json")}


@pytest.mark.parametrize("plan", list(LARGE_PLANS))
def test_large_workload_32_slices_vs_einsum_oracle(qx, plan):
    """6x6 depth-14 workload, bench launch configuration, slices 0..31, under the seeded greedy plan,
    the local-search plan and the annealed plan the benchmark runs (which slices other bonds: its
    slices 0..31 are other sub-networks, with their own golden partial sum)."""
    fn, gname = LARGE_PLANS[plan]
    w = getattr(W, fn)()
    g, ref = _golden_large(gname)
    from tests.golden.make_large_golden import plan_digest
    assert g["plan_sha256"] == plan_digest(w), "planner output changed; regenerate the golden file"
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 1)
    got = c.contract_slices(w.bitstrings, 0, 32)[0]
    assert_parity(got, ref)
    # one slice recomputed by the oracle in the test itself
    one = oe.contract_once(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 7, w.bitstrings[0])
    assert_parity(c.contract_slices(w.bitstrings, 7, 8)[0], one)


@pytest.mark.parametrize("rows,cols,depth,n_open,n_slice,n_bits", [
    (3, 3, 8, 3, 2, 5), (2, 5, 10, 0, 4, 33), (3, 4, 6, 2, 3, 1), (4, 4, 8, 4, 5, 7), (2, 4, 6, 8, 0, 2)])
def test_persistent_executor_vs_statevector(qx, rows, cols, depth, n_open, n_slice, n_bits):
    circ, om, order, sliced, bits = grid_case(rows, cols, depth, 31 + depth, n_open, n_slice, n_bits)
    recs = C.gates_to_records(circ)
    ref = oracle.sv_amplitudes(circ.n_qubits, recs, om, bits)
    p = _contractor(qx, circ, om, order, sliced, n_bits, executor=qx.EXEC_PERSISTENT)
    b = _contractor(qx, circ, om, order, sliced, n_bits, executor=qx.EXEC_BATCHED)
    if n_open == circ.n_qubits and n_slice == 0:
        # nothing depends on the pair: the persistent executor does not apply
        with pytest.raises(qx.QXError):
            p.contract(bits)
        return
    gp = p.contract(bits)
    gb = b.contract(bits)
    assert_parity(gp, ref)
    assert rel_l2(gp, gb) <= 1e-6


def test_persistent_executor_on_sliced_workload(qx):
    w = W.sliced()
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings),
                      executor=qx.EXEC_PERSISTENT)
    qx.qx_set_profiling(c.h, True)
    got = c.contract(w.bitstrings)
    prof = qx.qx_profile_read(c.h)
    assert prof["persist"]["launches"] == 2  # one launch for the invariant tensors, one for all pairs
    assert_parity(got, ref)


def test_sharded_slices_single_rank_group(qx):
    import datetime
    import socket

    import torch.distributed as dist

    from paper_2110_09894_gb300.dist import sharded_amplitudes
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            timeout=datetime.timedelta(seconds=30))
    try:
        circ, om, order, sliced, bits = grid_case(3, 4, 8, 23, 2, 4, 3)
        c = _contractor(qx, circ, om, order, sliced, 3)
        got = sharded_amplitudes(c, bits, 0, 1)
        assert rel_l2(got, c.contract(bits)) < 1e-15
    finally:
        dist.destroy_process_group()


def test_graph_replay_matches_eager_and_follows_new_data(qx):
    import torch
    circ, om, order, sliced, bits = grid_case(3, 4, 8, 44, 1, 3, 6)
    c = _contractor(qx, circ, om, order, sliced, 6)
    d_bits = torch.from_numpy(bits).cuda()
    out = torch.empty((6, 2, 2), dtype=torch.float64, device="cuda")
    runs = []
    for _ in range(3):  # eager, capture + launch, replay
        c.contract_device(d_bits, out)
        torch.cuda.synchronize()
        runs.append(out.cpu().numpy().copy())
    assert np.array_equal(runs[0], runs[1]) and np.array_equal(runs[1], runs[2])
    # new bitstrings in the same buffer: the replayed graph reads them
    bits2 = C.random_bitstrings(circ.n_qubits, 6, 99)
    d_bits.copy_(torch.from_numpy(bits2))
    c.contract_device(d_bits, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle.sv_amplitudes(circ.n_qubits, C.gates_to_records(circ), om, bits2)
    assert_parity(got[..., 0] + 1j * got[..., 1], ref)
    qx.qx_set_graphs(c.h, False)
    c.contract_device(d_bits, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), got)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_concurrent_issue_is_bit_identical_to_in_order(qx, precision):
    """Steps issued over several streams along the dependency lists give the same bits as in order."""
    import torch
    w = W.sliced()
    st = torch.cuda.Stream()
    runs = {}
    for n_streams, max_items in ((1, 0), (8, 0), (3, 0), (1, 1000), (8, 1000)):
        c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings),
                          precision=precision, max_items=max_items, stream=st)
        qx.qx_set_streams(c.h, n_streams)
        d_bits = torch.from_numpy(w.bitstrings).cuda()
        out = torch.empty((len(w.bitstrings), 1, 2), dtype=torch.float64, device="cuda")
        got = []
        for _ in range(3):  # eager, graph capture + launch, replay
            with torch.cuda.stream(st):
                c.contract_device(d_bits, out)
            st.synchronize()
            got.append(out.cpu().numpy().copy())
        assert np.array_equal(got[0], got[1]) and np.array_equal(got[1], got[2])
        if max_items:
            assert c.stats()["batches"] > 1
        runs[(n_streams, max_items)] = got[0]
        c.close()
    assert np.array_equal(runs[(8, 0)], runs[(1, 0)])
    assert np.array_equal(runs[(3, 0)], runs[(1, 0)])
    assert np.array_equal(runs[(8, 1000)], runs[(1, 1000)])
    if precision <= 2:
        ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
        got = runs[(8, 0)][..., 0] + 1j * runs[(8, 0)][..., 1]
        assert_parity(got, ref)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_slice_level_is_bit_identical_to_per_pair(qx, precision):
    """Steps that no output bit touches, run once per slice and read by every bitstring of the slice,
    give the bits the per-pair execution gives (same kernels, same operands), with less work."""
    import torch
    w = W.sliced()
    d_bits = torch.from_numpy(w.bitstrings).cuda()
    runs, flops = {}, {}
    for off, max_items in ((0, 0), (1, 0), (0, 700), (0, 100)):
        c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings),
                          precision=precision, max_items=max_items, no_slice_level=off)
        out = c.contract_device(d_bits)
        torch.cuda.synchronize()
        runs[(off, max_items)] = out.cpu().numpy()
        flops[(off, max_items)] = c.stats()["flops"]
        c.close()
    assert np.array_equal(runs[(0, 0)], runs[(1, 0)])
    assert np.array_equal(runs[(0, 700)], runs[(1, 0)])  # 2 slices per batch
    assert np.array_equal(runs[(0, 100)], runs[(1, 0)])  # fewer pairs per batch than bitstrings
    assert flops[(0, 0)] < 0.5 * flops[(1, 0)]


@pytest.mark.parametrize("rows,cols,depth,n_open,n_slice,n_bits,max_items", [
    (3, 4, 8, 1, 4, 6, 7), (3, 4, 8, 1, 4, 6, 13), (4, 4, 8, 0, 5, 9, 0), (3, 3, 8, 9, 3, 2, 0),
    (2, 5, 10, 2, 4, 33, 50)])
def test_slice_level_vs_statevector(qx, rows, cols, depth, n_open, n_slice, n_bits, max_items):
    # ragged batches: a batch may hold one slice and part of the bitstrings, several slices, or (all
    # qubits open) no output bit at all, so the root itself is per slice
    circ, om, order, sliced, bits = grid_case(rows, cols, depth, 90 + depth + n_bits, n_open, n_slice, n_bits)
    ref = oracle.sv_amplitudes(circ.n_qubits, C.gates_to_records(circ), om, bits)
    for prec in (0, 1):
        c = _contractor(qx, circ, om, order, sliced, n_bits, precision=prec, max_items=max_items)
        got = c.contract(bits)
        assert_parity(got, ref)
        c.close()


def test_memoised_invariants_give_the_same_bits(qx):
    """qx_set_memo: later calls skip the invariant steps and read the kept tensors; new bitstrings,
    graph replay and the static-scratch entry point in between all give the bits of fresh calls."""
    import torch
    w = W.sliced()
    bits_a = torch.from_numpy(w.bitstrings).cuda()
    bits_b = torch.from_numpy(C.random_bitstrings(w.n_qubits, len(w.bitstrings), 4242)).cuda()
    fresh = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings), precision=1)
    want_a = fresh.contract_device(bits_a).cpu().numpy()
    want_b = fresh.contract_device(bits_b).cpu().numpy()
    full_flops = fresh.stats()["flops"]
    fresh.close()
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings), precision=1)
    qx.qx_set_memo(c.h, 1)
    out = torch.empty((len(w.bitstrings), 1, 2), dtype=torch.float64, device="cuda")
    for i in range(4):  # eager with the invariant steps, eager without, graph capture, replay
        c.contract_device(bits_a, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), want_a), i
        if i == 1:
            assert c.stats()["flops"] < full_flops
    assert np.array_equal(c.contract_device(bits_b).cpu().numpy(), want_b)
    d_static = torch.empty_like(out)
    qx.qx_contract_device_static(c.h, bits_b.data_ptr(), len(w.bitstrings), d_static.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(d_static.cpu().numpy(), want_b)
    c.contract_device(bits_a, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want_a)
    with pytest.raises(qx.QXError):
        qx.qx_set_memo(c.h, 2)
    c.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("plan", ["sliced_level_aware", "sliced_checkpoint"])
def test_level_aware_plan_vs_statevector(qx, precision, plan):
    # the sliced workload's circuit under the plans chosen for executed flops per call
    w = getattr(W, plan)()
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings), precision=precision)
    got = c.contract(w.bitstrings)
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
    assert_parity(got, ref)
    assert c.stats()["flops"] == w.meta["executed_flops"]
    c.close()


def test_stream_count_is_checked(qx):
    circ, om, order, sliced, bits = grid_case(3, 3, 6, 5, 1, 1, 2)
    c = _contractor(qx, circ, om, order, sliced, 2)
    for bad in (0, 33, -1):
        with pytest.raises(qx.QXError):
            qx.qx_set_streams(c.h, bad)
    qx.qx_set_streams(c.h, 32)
    ref = oracle.sv_amplitudes(circ.n_qubits, C.gates_to_records(circ), om, bits)
    assert_parity(c.contract(bits), ref)


def test_edge_cases(qx):
    # no bitstrings
    circ, om, order, sliced, bits = grid_case(2, 3, 4, 61, 1, 2, 3)
    c = _contractor(qx, circ, om, order, sliced, 3)
    with pytest.raises(qx.QXError) as e:
        c.contract(np.zeros((0, circ.n_qubits), np.uint8))
    assert e.value.code == qx.QX_EINVAL
    # bytes at open qubits are ignored
    b2 = bits.copy()
    b2[:, -1] ^= 1
    assert np.array_equal(c.contract(bits), c.contract(b2))
    # disconnected network: two qubits without a two-qubit gate (outer product step)
    d = C.Circuit(2)
    d.append((0,), C.SQRT_X)
    d.append((1,), C.SQRT_W)
    from qxgen.workloads import make_plan
    om2 = np.array([0, 1], np.uint8)
    order2, sliced2, _, _ = make_plan(d, om2, 0, 3)
    cc = _contractor(qx, d, om2, order2, sliced2, 2)
    bb = np.array([[0, 0], [1, 0]], np.uint8)
    got = cc.contract(bb)
    ref = oracle.sv_amplitudes(2, C.gates_to_records(d), om2, bb)
    assert_parity(got, ref)
    # every qubit closed but the plan slices the only bond of a one-gate circuit
    e1 = C.Circuit(1)
    e1.append((0,), C.SQRT_Y)
    ce = _contractor(qx, e1, np.zeros(1, np.uint8), [(0, 1), (2, 3)], [0], 2)
    got = ce.contract(np.array([[0], [1]], np.uint8))[:, 0]
    assert np.allclose(got, C.SQRT_Y[:, 0], atol=1e-7)


@pytest.mark.parametrize("executor", [1, 2])
def test_device_slice_sum_is_compensated(qx, executor):
    """The FP64 cross-slice sum on the device (Eq. 2) is compensated: slice results X, 1, -X, -1
    (X = 2^60, exact in FP32) must sum to exactly 0 = math.fsum of the oracle's per-slice values; a
    plain running FP64 sum would give -1 (the CPU pin of this case shows that)."""
    from ._util import cancelling_slices_case
    circ, om, order, sliced, bits = cancelling_slices_case()
    recs = C.gates_to_records(circ)
    per = [oe.amplitudes(2, recs, om, order, sliced, bits, slices=[s])[0, 0] for s in range(4)]
    want = complex(math.fsum(p.real for p in per), math.fsum(p.imag for p in per))
    for max_items in (0, 1):  # all four slices in one batch, or one slice per batch
        c = _contractor(qx, circ, om, order, sliced, 1, executor=executor, max_items=max_items)
        got = c.contract(bits)[0, 0]
        assert got == want, (got, want)
        c.close()


def test_bitstring_batches_reuse_the_slice_results(qx):
    """When a slice's bitstrings need several batches of the per-pair region (max_items below the number
    of bitstrings), the later batches run only the per-pair steps and read the per-slice results the
    first batch left in the per-slice region: amplitudes as the single-batch call's."""
    w = W.sliced_level_aware()
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
    full = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings), precision=1)
    a = full.contract(w.bitstrings)
    full.close()
    for cap in (100, 7):
        c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings), precision=1,
                          max_items=cap)
        assert "slice" in {ln.split()[3] for ln in qx.qx_describe_plan(c.h).splitlines()}
        got = c.contract(w.bitstrings)
        assert c.stats()["batches"] > w.n_slices  # several bitstring batches per slice
        assert_parity(got, ref)
        assert rel_l2(got, a) < 1e-6
        c.close()
