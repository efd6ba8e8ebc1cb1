"""The level-aware plan choice (host logic, no GPU).

executed_cost models what the batched executor runs per call: invariant steps
once, per-slice steps once per slice, the rest per (slice, bitstring) pair.
It is checked against the library's own compiled plan (the step sizes and
levels qx_describe_plan lists, an independent computation in the C++ plan
compiler), and the plan it selects is checked to compute the right amplitude
with the einsum oracle against the state vector.
"""
import re

import numpy as np
import pytest

import oracle
from oracle import einsum as oe
from qxgen import workloads as W
from qxgen.plan import executed_cost, network_legs, plan_cost


def _legs(w):
    legs, _, open_edges = network_legs(w.n_qubits, [g.qubits for g in w.circuit.gates], w.open_mask)
    return legs, w.n_qubits - len(open_edges)


def _library_executed(qx, w, n_bits):
    h = qx.qx_create(-1, precision=1)
    try:
        qx.qx_build_network(h, w.n_qubits, w.gates, w.open_mask)
        qx.qx_set_plan(h, w.order, w.sliced)
        total = 0
        for line in qx.qx_describe_plan(h).splitlines():
            f = line.split()
            m = re.search(r" m=(\d+) k=(\d+) n=(\d+)", line)
            if not m:
                continue  # permutes move data only
            flops = 8 * (1 << (int(m.group(1)) + int(m.group(2)) + int(m.group(3))))
            mult = {"pair": w.n_slices * n_bits, "slice": w.n_slices, "shared": 1}[f[3]]
            total += flops * mult
        return total
    finally:
        qx.qx_destroy(h)


@pytest.fixture(scope="module")
def qx():
    from paper_2110_09894_gb300 import build
    build.build()
    from paper_2110_09894_gb300 import qx as mod
    return mod


@pytest.mark.parametrize("name", ["sliced", "sliced_level_aware", "sliced_checkpoint"])
def test_executed_cost_matches_the_compiled_plan(qx, name):
    w = getattr(W, name)()
    legs, n_out = _legs(w)
    assert executed_cost(legs, w.order, w.sliced, n_out, 256) == _library_executed(qx, w, 256)


def test_level_aware_plan_executes_less_at_the_same_peak():
    base, lvl = W.sliced(), W.sliced_level_aware()
    legs, n_out = _legs(base)
    e0 = executed_cost(legs, base.order, base.sliced, n_out, 256)
    e1 = executed_cost(legs, lvl.order, lvl.sliced, n_out, 256)
    assert e1 < 0.6 * e0
    assert lvl.peak_rank <= base.peak_rank and len(lvl.sliced) == len(base.sliced)
    assert e1 == lvl.meta["executed_flops"]


def test_level_aware_plan_gives_the_state_vector_amplitude():
    w = W.sliced_level_aware()
    bits = w.bitstrings[:1]
    got = oe.amplitudes(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, bits)
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, bits)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-13)


def test_checkpoint_plan_executes_a_fraction_at_the_same_peak():
    # the stored plan (level-aware choice improved by local search): each slice's environment is
    # contracted once, every bitstring adds little
    base, ck = W.sliced(), W.sliced_checkpoint()
    legs, n_out = _legs(base)
    assert ck.peak_rank <= base.peak_rank and list(ck.sliced) and len(ck.sliced) == len(base.sliced)
    assert executed_cost(legs, ck.order, ck.sliced, n_out, 256) < 0.05 * executed_cost(legs, base.order, base.sliced,
                                                                                        n_out, 256)


def test_checkpoint_plan_gives_the_state_vector_amplitude():
    w = W.sliced_checkpoint()
    bits = w.bitstrings[:2]
    got = oe.amplitudes(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, bits)
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, bits)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-13)


def test_tree_rotation_round_trip_and_local_search_only_improves():
    from qxgen.plan import _order_to_tree, _tree_to_order, local_search_plan
    w = W.small()
    legs, n_out = _legs(w)
    ch, root = _order_to_tree(len(legs), w.order)
    order = _tree_to_order(len(legs), ch, root)
    assert executed_cost(legs, order, w.sliced, n_out, 16) == executed_cost(legs, w.order, w.sliced, n_out, 16)
    o2, cost, _ = local_search_plan(legs, w.order, w.sliced, n_out, 16, max_peak=w.peak_rank, iters=300, seed=3)
    assert cost <= executed_cost(legs, w.order, w.sliced, n_out, 16)
    assert cost == executed_cost(legs, o2, w.sliced, n_out, 16)
    got = oe.amplitudes(w.n_qubits, w.gates, w.open_mask, o2, w.sliced, w.bitstrings[:3])
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings[:3])
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-13)


def test_local_search_is_deterministic_for_a_seed():
    from qxgen.plan import local_search_plan
    w = W.small()
    legs, n_out = _legs(w)
    a = local_search_plan(legs, w.order, w.sliced, n_out, 16, max_peak=w.peak_rank, iters=200, seed=5)
    b = local_search_plan(legs, w.order, w.sliced, n_out, 16, max_peak=w.peak_rank, iters=200, seed=5)
    assert a == b


def test_stored_plan_is_checked_against_its_circuit(monkeypatch):
    W.sliced_checkpoint.cache_clear()
    monkeypatch.setattr(W, "circuit_digest", lambda circ: "0" * 64)
    with pytest.raises(ValueError):
        W.sliced_checkpoint()
    monkeypatch.undo()
    W.sliced_checkpoint.cache_clear()
    assert W.sliced_checkpoint().meta["executed_flops"] > 0


def test_large_local_search_plan_keeps_the_slices_and_its_golden_agrees():
    """The stored local-search plan of the large workload slices the same bonds and stays within the
    2^28 peak; the oracle's 32-slice partial sums under the two orders (two golden files written by
    tests/golden/make_large_golden.py) agree to complex128 rounding: the order changes only the
    rounding (Sec. III-A), slicing fixes which sub-networks are summed (Eq. 2)."""
    import json
    import os
    w0, w1 = W.large(), W.large_local_search()
    assert w1.sliced == list(w0.sliced) and w1.peak_rank <= 28
    assert w1.meta["executed_flops"] < executed_cost(*_legs(w0)[:1], w0.order, w0.sliced, _legs(w0)[1], 1) / 10
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    g = [json.load(open(os.path.join(here, n))) for n in ("large_slices0_31.json", "large_ls_slices0_31.json")]
    a, b = (np.array(x["re"]) + 1j * np.array(x["im"]) for x in g)
    assert g[0]["bitstring"] == g[1]["bitstring"]
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-12


def test_large_annealed_plan_and_its_golden_follow_eq2():
    """The stored annealed plan of the large workload slices 10 distinct bonds the library accepts
    (1024 slices), keeps every intermediate within 2^24 entries and executes fewer flops per call than
    the local-search plan it started from.  Its golden file (the oracle's partial sum over slices
    0..31, written by tests/golden/make_large_golden.py) carries its digest, and by Eq. 2 equals one
    oracle contraction in which the five sliced bonds that slices 0..31 vary are left whole and the
    other five are fixed to 0: summing a bond's slices is not slicing it."""
    import json
    import os
    from qxgen.plan import sliceable_bonds
    from tests.golden.make_large_golden import plan_digest
    w, w0 = W.large_annealed(), W.large_local_search()
    legs, n_out = _legs(w)
    _, _, open_edges = network_legs(w.n_qubits, [g.qubits for g in w.circuit.gates], w.open_mask)
    assert len(w.sliced) == 10 and len(set(w.sliced)) == 10 and w.n_slices == 1024
    assert set(w.sliced) <= set(sliceable_bonds(legs, n_out, open_edges)) and w.peak_rank <= 24
    assert set(w.sliced) != set(w0.sliced)
    assert w.meta["executed_flops"] < w0.meta["executed_flops"]
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    with open(os.path.join(here, "large_sa_slices0_31.json")) as f:
        g = json.load(f)
    assert g["plan_sha256"] == plan_digest(w) and g["slices"] == [0, 32]
    ref = np.array(g["re"]) + 1j * np.array(g["im"])
    whole = oe.amplitudes(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced[5:], w.bitstrings, slices=[0])[0]
    assert np.linalg.norm(whole - ref) / np.linalg.norm(ref) < 1e-12


def test_anneal_plan_keeps_the_slice_count_and_finds_a_cheaper_plan():
    """anneal_plan on the 20-qubit sliced circuit (six sliced bonds, executed flops as the cost): the
    result slices six distinct sliceable bonds, fits the peak, costs no more than the start, and the
    einsum oracle under it reproduces the state vector (any order and any sliced set give the same
    amplitudes, Eq. 2)."""
    from qxgen.plan import anneal_plan, plan_cost, sliceable_bonds
    w = W.sliced()
    legs, n_out = _legs(w)
    _, _, open_edges = network_legs(w.n_qubits, [g.qubits for g in w.circuit.gates], w.open_mask)
    cands = sliceable_bonds(legs, n_out, open_edges)
    nb = 4
    start = executed_cost(legs, w.order, w.sliced, n_out, nb)
    order, sliced, cost, acc = anneal_plan(legs, w.order, w.sliced, n_out, nb, 16, 600, 5, executed_cost,
                                           cands, p_swap=0.3)
    # the same seed gives the same plan (plans are inputs written once and checked on load)
    assert anneal_plan(legs, w.order, w.sliced, n_out, nb, 16, 600, 5, executed_cost, cands, p_swap=0.3) == \
        (order, sliced, cost, acc)
    assert len(sliced) == len(w.sliced) and len(set(sliced)) == len(sliced) and set(sliced) <= set(cands)
    assert plan_cost(legs, order, sliced)[0] <= 16 and acc > 0
    assert cost == executed_cost(legs, order, sliced, n_out, nb) <= start
    bits = w.bitstrings[:nb]
    ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, bits)
    got = oe.amplitudes(w.n_qubits, w.gates, w.open_mask, order, sliced, bits)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10


def test_sweep_order_contracts_the_network_with_the_qubit_count_as_peak():
    """sweep_order on grid circuits with and without open qubits and sliced bonds: a full SSA order
    (every tensor used once), no intermediate above n legs, every step below the final layer
    independent of the bitstring, and the einsum oracle under it reproduces the state vector."""
    from qxgen.plan import sweep_order
    from tests._util import grid_case
    from qxgen import circuits as C
    for rows, cols, depth, n_open, n_slice, n_bits, seed in ((3, 3, 8, 0, 0, 5, 1), (3, 4, 6, 2, 2, 3, 2),
                                                             (2, 5, 9, 0, 1, 4, 3)):
        circ, om, _, sliced, bits = grid_case(rows, cols, depth, seed, n_open, n_slice, n_bits)
        gq = [g.qubits for g in circ.gates]
        legs, _, open_edges = network_legs(circ.n_qubits, gq, om)
        n_out = circ.n_qubits - len(open_edges)
        order = sweep_order(legs, circ.n_qubits, n_out, gq)
        n = len(legs)
        used = [x for p in order for x in p]
        assert len(order) == n - 1 and sorted(used) == list(range(2 * n - 2))
        assert plan_cost(legs, order)[0] <= circ.n_qubits
        recs = C.gates_to_records(circ)
        ref = oracle.sv_amplitudes(circ.n_qubits, recs, om, bits)
        got = oe.amplitudes(circ.n_qubits, recs, om, order, sliced, bits)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
    # a closed qubit that no gate touches: its output vector meets its input directly
    circ = C.random_grid_circuit(1, 3, 4, 7)
    gq = [g.qubits for g in circ.gates]
    om = np.zeros(4, np.uint8)
    legs, _, _ = network_legs(4, gq, om)
    order = sweep_order(legs, 4, 4, gq)
    recs = C.gates_to_records(circ)
    bits = C.random_bitstrings(4, 3, 1)
    ref = oracle.sv_amplitudes(4, recs, om, bits)
    assert np.abs(oe.amplitudes(4, recs, om, order, [], bits) - ref).max() < 1e-12
    # the steps that reach an output bit (their subtree holds an output vector) come last, after every
    # bitstring-independent step; without sliced bonds a bitstring then adds a small part of a call
    circ, om, _, _, _ = grid_case(3, 4, 12, 4, 0, 0, 1)
    gq = [g.qubits for g in circ.gates]
    legs, _, open_edges = network_legs(circ.n_qubits, gq, om)
    n = len(legs)
    order = sweep_order(legs, circ.n_qubits, circ.n_qubits, gq)
    reach = [t >= n - circ.n_qubits for t in range(n)]
    for a, b in order:
        reach.append(reach[a] or reach[b])
    steps = reach[n:]
    first = steps.index(True)
    assert all(steps[first:]) and first > len(steps) // 2
    one, many = executed_cost(legs, order, [], circ.n_qubits, 1), executed_cost(legs, order, [], circ.n_qubits, 64)
    assert (many - one) / 63 < one / 4


def test_batched_annealed_plans_keep_their_circuits_slices_and_peak():
    """The annealed plans of the batched workload's heaviest circuits (qxgen/plans/batched_annealed.json)
    replace their stored plans: each keeps its circuit's drawn number of sliced bonds (distinct bonds the
    library accepts), every intermediate within 2^28 entries, and its recorded launch-list estimate is
    below the stored plan's; the library compiles each (host-only handle) and the compiled launch list
    stays ordered with every read and write.  Their amplitudes are checked against the state vectors on
    the GPU (the 256-circuit test)."""
    import json
    import os
    from qxgen.plan import sliceable_bonds
    from paper_2110_09894_gb300 import qx
    from tests.test_plan_deps import _check, _parse, _plan_lines
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "qxgen", "plans",
                        "batched_annealed.json")
    with open(path) as f:
        plans = json.load(f)["plans"]
    assert len(plans) >= 5
    specs = W.batched_specs()
    for d in plans:
        j = d["j"]
        w, w0 = W.batched_circuit(j), W.batched_circuit(j, annealed=False)
        assert [tuple(p) for p in d["order"]] == list(w.order) and list(w.sliced) == d["sliced"]
        legs, n_out = _legs(w)
        _, _, open_edges = network_legs(w.n_qubits, [g.qubits for g in w.circuit.gates], w.open_mask)
        assert len(w.sliced) == specs[j][2] == len(w0.sliced) and len(set(w.sliced)) == len(w.sliced)
        assert set(w.sliced) <= set(sliceable_bonds(legs, n_out, open_edges)) and w.peak_rank <= 28
        assert d["estimated_s"] < d["stored_estimated_s"]
        _check(_parse(_plan_lines(qx, w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 1)))


def test_executed_time_reduces_to_executed_flops_with_one_rate():
    """With every kernel family at one rate, unbounded memory bandwidth and no launch cost, the time
    estimate is the executed flops over that rate (the same levels and multiplicities); the memory
    term alone grows with the bytes a plan moves."""
    from qxgen.plan import executed_time
    for w in (W.small(), W.sliced()):
        legs, n_out = _legs(w)
        one = {"tc": 1e12, "gemm": 1e12, "gather": 1e12, "hbm": float("inf"), "launch": 0.0}
        t = executed_time(legs, w.order, w.sliced, n_out, len(w.bitstrings), rates=one)
        f = executed_cost(legs, w.order, w.sliced, n_out, len(w.bitstrings))
        assert abs(t * 1e12 - f) <= 1e-9 * f
        mem = {"tc": float("inf"), "gemm": float("inf"), "gather": float("inf"), "hbm": 1.0, "launch": 0.0}
        assert executed_time(legs, w.order, w.sliced, n_out, len(w.bitstrings), rates=mem) > 0
