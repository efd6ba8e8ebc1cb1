"""Dependency lists of the compiled plan (host logic, no GPU).

Launches issued over several streams must keep every pair of conflicting
launches in plan order: if two launches touch overlapping storage of the same
region and at least one of them writes it (or both use the tensor-core scale
words), the later one must be reachable from the earlier one through the
dependency lists.  Then any order the streams pick reads the same data as the
in-order execution.  The storages and lists come from qx_describe_plan.
"""
import re

import pytest

from qxgen import workloads as W
from tests._util import grid_case
from qxgen import circuits as C


def _plan_lines(qx, n, gates, om, order, sliced, precision):
    h = qx.qx_create(-1, precision=precision)
    try:
        qx.qx_build_network(h, n, gates, om)
        qx.qx_set_plan(h, order, sliced)
        return qx.qx_describe_plan(h).splitlines()
    finally:
        qx.qx_destroy(h)


def _parse(lines):
    ops = []
    for i, line in enumerate(lines):
        assert line.startswith(f"{i} ")
        def ranges(key):
            m = re.search(key + r"=(\S*)", line)
            out = []
            for part in filter(None, m.group(1).split(",")):
                space, rest = part.split(":")
                off, n = rest.split("+")
                out.append((space, int(off), int(n)))
            return out
        after = re.search(r"after=(\S*)", line)
        deps = [int(x) for x in after.group(1).split(",")] if after and after.group(1) else []
        ops.append({"r": ranges("reads"), "w": ranges("writes"), "scale": " scale=1 " in line, "deps": deps})
    return ops


def _overlap(xs, ys):
    return any(a[0] == b[0] and a[1] < b[1] + b[2] and b[1] < a[1] + a[2] for a in xs for b in ys)


def _check(ops):
    anc = []
    for j, op in enumerate(ops):
        assert all(0 <= i < j for i in op["deps"])
        a = 0
        for i in op["deps"]:
            a |= anc[i] | (1 << i)
        anc.append(a)
    conflicts = 0
    for j, oj in enumerate(ops):
        for i in range(j):
            oi = ops[i]
            if (oi["scale"] and oj["scale"]) or _overlap(oi["w"], oj["r"]) or _overlap(oi["r"], oj["w"]) or \
                    _overlap(oi["w"], oj["w"]):
                conflicts += 1
                assert (anc[j] >> i) & 1, f"op {j} is not ordered after conflicting op {i}"
    return conflicts


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
def test_conflicting_launches_stay_ordered_on_the_sliced_workload(precision):
    from paper_2110_09894_gb300 import qx
    w = W.sliced()
    ops = _parse(_plan_lines(qx, w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, precision))
    assert _check(ops) > len(ops)  # space is reused: many conflicts, all ordered
    # producers precede consumers: each storage read by a launch was written by an earlier one
    for j, op in enumerate(ops):
        for r in op["r"]:
            assert any(_overlap([r], ops[i]["w"]) for i in range(j))


@pytest.mark.parametrize("seed", [3, 8])
def test_conflicting_launches_stay_ordered_on_grid_plans(seed):
    from paper_2110_09894_gb300 import qx
    circ, om, order, sliced, _ = grid_case(4, 4, 10, seed, 2, 3, 1)
    for precision in (0, 3):
        ops = _parse(_plan_lines(qx, circ.n_qubits, C.gates_to_records(circ), om, order, sliced, precision))
        _check(ops)


def test_dependency_check_catches_a_missing_edge():
    """A plan listing with one dependency removed fails the check (the check is not vacuous)."""
    from paper_2110_09894_gb300 import qx
    w = W.sliced()
    ops = _parse(_plan_lines(qx, w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 0))
    j = next(j for j in range(len(ops) - 1, 0, -1) if ops[j]["deps"])
    ops[j]["deps"] = ops[j]["deps"][:-1]
    with pytest.raises(AssertionError):
        _check(ops)


def test_per_slice_launches_read_no_per_pair_storage():
    """Steps that no output bit touches run once per slice: they may read invariant and per-slice
    tensors only, and every per-pair launch comes after the per-slice launches it reads."""
    from paper_2110_09894_gb300 import qx
    w = W.sliced()
    lines = _plan_lines(qx, w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 1)
    ops = _parse(lines)
    levels = [line.split()[3] for line in lines]
    assert levels.count("slice") >= 5 and levels.count("pair") >= 5
    for j, (op, lv) in enumerate(zip(ops, levels)):
        for space, _, _ in op["w"]:
            assert space == {"shared": "shared", "slice": "slice", "pair": "pair"}[lv]
        if lv != "pair":
            assert all(space != "pair" for space, _, _ in op["r"])
        if lv == "shared":
            assert all(space == "shared" for space, _, _ in op["r"])
    _check(ops)


def test_per_slice_level_shrinks_work_and_workspace():
    from paper_2110_09894_gb300 import qx
    w = W.sliced()
    got = {}
    for off in (0, 1):
        h = qx.qx_create(-1, precision=1, no_slice_level=off)
        qx.qx_build_network(h, w.n_qubits, w.gates, w.open_mask)
        qx.qx_set_plan(h, w.order, w.sliced)
        got[off] = qx.qx_workspace_size(h, len(w.bitstrings), w.n_slices * len(w.bitstrings))
        qx.qx_destroy(h)
    assert got[0] < 0.6 * got[1]
    with pytest.raises(qx.QXError):
        qx.qx_create(-1, no_slice_level=2)


def _chains(lines):
    out = []
    for line in lines:
        m = re.search(r" chain=(\d+)", line)
        out.append(int(m.group(1)) if m else -1)
    return out


def _check_chains(ops, chains):
    """Prologue chains run on different CTAs with no synchronisation: steps of different chains must
    touch no common storage where either writes, and a step's dependencies on other prologue steps
    must sit in its own chain (which runs them earlier, in plan order)."""
    for j, cj in enumerate(chains):
        if cj < 0:
            continue
        for i in ops[j]["deps"]:
            if chains[i] >= 0:
                assert chains[i] == cj, f"step {j} (chain {cj}) depends on step {i} of chain {chains[i]}"
        for i in range(j):
            ci = chains[i]
            if ci < 0 or ci == cj:
                continue
            oi, oj = ops[i], ops[j]
            assert not (_overlap(oi["w"], oj["r"]) or _overlap(oi["r"], oj["w"]) or _overlap(oi["w"], oj["w"])), \
                f"steps {i} (chain {ci}) and {j} (chain {cj}) share storage"


@pytest.mark.parametrize("precision", [0, 1])
def test_prologue_chains_share_no_storage(precision):
    from paper_2110_09894_gb300 import qx
    w = W.sliced()
    lines = _plan_lines(qx, w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, precision)
    ops, chains = _parse(lines), _chains(lines)
    levels = [line.split()[3] for line in lines]
    # every invariant step of this plan is small: all of them run in the one prologue launch
    assert all((c >= 0) == (lv == "shared") for c, lv in zip(chains, levels))
    assert len(set(c for c in chains if c >= 0)) > 10
    _check_chains(ops, chains)


def test_chain_check_catches_a_step_in_the_wrong_chain():
    from paper_2110_09894_gb300 import qx
    w = W.sliced()
    lines = _plan_lines(qx, w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 0)
    ops, chains = _parse(lines), _chains(lines)
    j = next(j for j in range(len(ops)) if chains[j] >= 0 and any(chains[i] >= 0 for i in ops[j]["deps"]))
    chains[j] = max(chains) + 1
    with pytest.raises(AssertionError):
        _check_chains(ops, chains)


def test_in_place_a_steps_of_the_36_qubit_plan():
    """The resident-B' direct steps that read A where it is stored (no permute before them): each
    lists the address position of every K bit and row bit of A, together every position of A once;
    the 128-row x 16-K tile of a stage starts with a run of at least 8 positions (at most 8
    contiguous blocks), and the launch list stays ordered with those reads."""
    from paper_2110_09894_gb300 import qx
    w = W.large_local_search()
    lines = _plan_lines(qx, w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 1)
    gathered = [line for line in lines if " a_gather=1" in line]
    assert len(gathered) >= 3
    ops = _parse(lines)
    for line in gathered:
        f = dict(x.split("=", 1) for x in line.split()[4:] if "=" in x)
        assert line.split()[2] == "tc_direct"
        mb, kb, nb = int(f["m"]), int(f["k"]), int(f["n"])
        ak = [int(x) for x in f["ak"].split(",")]
        am = [int(x) for x in f["am"].split(",")]
        assert len(ak) == kb and len(am) == mb and sorted(ak + am) == list(range(mb + kb))
        tile = sorted(am[:7] + ak[:4])
        run = 0
        while run < 11 and tile[run] == run:
            run += 1
        assert run >= 8
        assert nb in (5, 6)  # one B tile: the resident-B' kernel
        # A comes straight from the step that produced it, not from a permute
        i = int(line.split()[0])
        a_read = ops[i]["r"][0]
        producers = [j for j in range(i) if _overlap([a_read], ops[j]["w"])]
        assert producers and lines[producers[-1]].split()[2] != "permute"
    _check(ops)


def _gather_invariants(lines):
    """Checks every in-place A step of a launch listing; returns how many there are."""
    ops = _parse(lines)
    n = 0
    for line in lines:
        if " a_gather=1" not in line:
            continue
        n += 1
        f = dict(x.split("=", 1) for x in line.split()[4:] if "=" in x)
        mb, kb = int(f["m"]), int(f["k"])
        ak = [int(x) for x in f["ak"].split(",")]
        am = [int(x) for x in f["am"].split(",")]
        assert sorted(ak + am) == list(range(mb + kb))
        tile = sorted(am[:7] + ak[:4])
        run = 0
        while run < 11 and tile[run] == run:
            run += 1
        assert run >= 8
        i = int(line.split()[0])
        producers = [j for j in range(i) if _overlap([ops[i]["r"][0]], ops[j]["w"])]
        assert producers and lines[producers[-1]].split()[2] != "permute"
    _check(ops)
    return n


def test_in_place_a_steps_of_the_batched_plans():
    """The same invariants over the stored plans of the uneven batch's heavy circuits (the ones the
    batched executor runs in 3xTF32)."""
    from paper_2110_09894_gb300 import qx
    total = 0
    for j in range(0, 256, 3):
        w = W.batched_circuit(j)
        if w.peak_rank <= 18 or w.n_qubits > 26:
            continue
        lines = _plan_lines(qx, w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 1)
        total += _gather_invariants(lines)
    assert total > 0


def test_launch_list_of_the_annealed_36_qubit_plan():
    """The benchmark's default plan (the annealed plan, which slices other bonds): its in-place A steps
    keep the invariants above and its launch list stays ordered with every read and write."""
    from paper_2110_09894_gb300 import qx
    w = W.large_annealed()
    lines = _plan_lines(qx, w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, 1)
    assert len(lines) > 100
    _gather_invariants(lines)
