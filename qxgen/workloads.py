"""The five synthetic workloads (seeded circuits, bitstrings and plans).

Seeds: circuit seed = 1000 * config + j (j = circuit number within the
config), bitstring seed = circuit seed + 500000, slicer / planner seed =
circuit seed + 700000.  The paper's own workloads are the Boixo random
circuits on qubit grids (Sec. IV-B); these seeded circuits stand in for them.

* small:   3x4 grid, depth 8, <0...0| and 16 random bitstrings, greedy plan,
           no slicing.
* sliced:  4x5 grid, depth 12, 6 sliced bonds (64 slices), 256 bitstrings.
* large:   6x6 grid, depth 14, 10 sliced bonds (1024 slices), qubits 30..35
           left open (64 amplitudes per contraction), peak <= 2^28 entries.
* batched: 256 circuits, n ~ U{16..28} on near-square grids, depth ~ U{8..16},
           S ~ U{0..8}, 1..64 bitstrings each, every one under its stored plan.
* serving: 32 circuits, n ~ U{20..40}, depth ~ U{10..16}, plans sliced until
           the peak intermediate fits 8 GB of complex64 (2^30 entries).
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, field

import numpy as np

from .circuits import (Circuit, SplitMix64, gates_to_records, near_square_shape, random_bitstrings,
                       random_grid_circuit)
from .plan import (executed_cost, greedy_order, level_aware_plan, network_legs, plan_cost, randomized_greedy,
                   tree_trim_slices)


@dataclass
class Workload:
    name: str
    circuit: Circuit
    open_mask: np.ndarray
    order: list
    sliced: list
    bitstrings: np.ndarray
    peak_rank: int = 0
    flops_per_slice: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_qubits(self):
        return self.circuit.n_qubits

    @property
    def gates(self):
        return gates_to_records(self.circuit)

    @property
    def n_open(self):
        return int(np.sum(self.open_mask))

    @property
    def n_slices(self):
        return 1 << len(self.sliced)

    def order_array(self):
        return np.asarray(self.order, dtype=np.int64).reshape(-1, 2)

    def sliced_array(self):
        return np.asarray(self.sliced, dtype=np.int64)


def make_plan(circ: Circuit, open_mask, n_slice, seed, trials=0, peak_rank=None, keep=12):
    legs, _, open_edges = network_legs(circ.n_qubits, [g.qubits for g in circ.gates], open_mask)
    # a qubit's final wire cannot be sliced: open ones are not bonds, closed ones carry the bitstring
    n_out = circ.n_qubits - len(open_edges)
    open_edges = list(open_edges) + [legs[t][0] for t in range(len(legs) - n_out, len(legs))]
    if trials:
        order, sliced = randomized_greedy(legs, trials, seed, n_slice, open_edges, keep=keep)
    else:
        order = greedy_order(legs)
        sliced = tree_trim_slices(legs, order, n_slice, seed, open_edges) if n_slice else []
    if peak_rank is not None:
        # keep slicing until the largest intermediate fits
        while plan_cost(legs, order, sliced)[0] > peak_rank:
            sliced = tree_trim_slices(legs, order, len(sliced) + 1, seed, open_edges)
    peak, flops = plan_cost(legs, order, sliced)
    return order, sliced, peak, flops


def _workload(name, circ, open_mask, n_slice, cseed, bits, trials=0, peak_rank=None, meta=None):
    order, sliced, peak, flops = make_plan(circ, open_mask, n_slice, cseed + 700000, trials, peak_rank)
    return Workload(name, circ, np.asarray(open_mask, np.uint8), order, sliced, bits, peak, flops, meta or {})


@functools.lru_cache(maxsize=None)
def small():
    cseed = 1001
    circ = random_grid_circuit(3, 4, 8, cseed)
    bits = np.concatenate([np.zeros((1, 12), np.uint8), random_bitstrings(12, 16, cseed + 500000)])
    return _workload("grid3x4_d8_amp17", circ, np.zeros(12, np.uint8), 0, cseed, bits)


@functools.lru_cache(maxsize=None)
def sliced():
    cseed = 2001
    circ = random_grid_circuit(4, 5, 12, cseed)
    bits = random_bitstrings(20, 256, cseed + 500000)
    return _workload("grid4x5_d12_s6_amp256", circ, np.zeros(20, np.uint8), 6, cseed, bits)


@functools.lru_cache(maxsize=None)
def sliced_level_aware():
    """The sliced workload's circuit, bitstrings and slice count with a plan chosen for the levels the
    executor runs steps at: seeded greedy candidates, each sliced by tree trimming, ranked by the flops
    one call of 256 bitstrings executes (executed_cost), peak kept at the default plan's 2^14."""
    cseed = 2001
    circ = random_grid_circuit(4, 5, 12, cseed)
    bits = random_bitstrings(20, 256, cseed + 500000)
    om = np.zeros(20, np.uint8)
    legs, _, open_edges = network_legs(20, [g.qubits for g in circ.gates], om)
    n_out = 20 - len(open_edges)
    no_slice = list(open_edges) + [legs[t][0] for t in range(len(legs) - n_out, len(legs))]
    order, sliced, executed, peak = level_aware_plan(legs, 40, cseed + 700000, 6, no_slice, n_out, len(bits),
                                                     max_peak=14)
    flops = plan_cost(legs, order, sliced)[1]
    return Workload("grid4x5_d12_s6_amp256_levelplan", circ, om, order, sliced, bits, peak, flops,
                    {"plan": "seeded greedy candidates ranked by executed flops per call (level-aware)",
                     "executed_flops": executed})


def circuit_digest(circ: Circuit) -> str:
    """sha256 of a circuit's gate records (identifies the circuit a stored plan was made for)."""
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(gates_to_records(circ)).tobytes()).hexdigest()


@functools.lru_cache(maxsize=None)
def sliced_checkpoint():
    """The sliced workload's circuit, bitstrings and slice count under the stored checkpoint plan
    (qxgen/plans/grid4x5_d12_s6_checkpoint.json, written by qxgen.make_plans): the level-aware plan
    improved by local search, so that each slice's environment is contracted once and every bitstring
    adds little work."""
    import json
    import os
    cseed = 2001
    circ = random_grid_circuit(4, 5, 12, cseed)
    bits = random_bitstrings(20, 256, cseed + 500000)
    om = np.zeros(20, np.uint8)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans", "grid4x5_d12_s6_checkpoint.json")
    with open(path) as f:
        d = json.load(f)
    if d["circuit_sha256"] != circuit_digest(circ):
        raise ValueError("stored plan was made for another circuit")
    order = [tuple(p) for p in d["order"]]
    sliced = list(d["sliced"])
    legs, _, open_edges = network_legs(20, [g.qubits for g in circ.gates], om)
    peak, flops = plan_cost(legs, order, sliced)
    executed = executed_cost(legs, order, sliced, 20 - len(open_edges), len(bits))
    if executed != d["executed_flops"] or peak > d["max_peak"]:
        raise ValueError("stored plan does not match its recorded cost")
    return Workload("grid4x5_d12_s6_amp256_checkpoint", circ, om, order, sliced, bits, peak, flops,
                    {"plan": "level-aware plan + local search (stored; checkpoint per slice)",
                     "executed_flops": executed})


def _load_stored_plan(fname, circ, open_mask, n_bits):
    """A plan stored in qxgen/plans/ (written by qxgen.make_plans), checked against the circuit it was
    made for and its recorded executed cost; returns (order, sliced, peak rank, flops per slice,
    executed flops per call, the record)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans", fname)
    with open(path) as f:
        d = json.load(f)
    if d["circuit_sha256"] != circuit_digest(circ):
        raise ValueError("stored plan was made for another circuit")
    order = [tuple(p) for p in d["order"]]
    sliced = list(d["sliced"])
    n = circ.n_qubits
    legs, _, open_edges = network_legs(n, [g.qubits for g in circ.gates], open_mask)
    peak, flops = plan_cost(legs, order, sliced)
    executed = executed_cost(legs, order, sliced, n - len(open_edges), n_bits)
    if executed != d["executed_flops"] or peak > d["max_peak"]:
        raise ValueError("stored plan does not match its recorded cost")
    return order, sliced, peak, flops, executed, d


@functools.lru_cache(maxsize=None)
def large_local_search():
    """The large workload (6x6 depth 14, qubits 30..35 open, the same 10 sliced bonds and bitstring)
    under its seeded plan improved by local search (qxgen/plans/grid6x6_d14_s10_open6_ls.json):
    the same 1024 slices, far fewer flops per slice, peak still <= 2^28 entries."""
    base = large()
    order, sliced, peak, flops, executed, d = _load_stored_plan("grid6x6_d14_s10_open6_ls.json", base.circuit,
                                                                base.open_mask, len(base.bitstrings))
    if sliced != list(base.sliced):
        raise ValueError("stored plan slices other bonds than the workload")
    return Workload("grid6x6_d14_s10_open6_ls", base.circuit, base.open_mask, order, sliced, base.bitstrings, peak,
                    flops, {"plan": "seeded greedy + tree trimming, then local search (stored)",
                            "executed_flops": executed, "made_by": d["made_by"]})


@functools.lru_cache(maxsize=None)
def large_annealed():
    """The large workload (6x6 depth 14, qubits 30..35 open, 10 sliced bonds, the same bitstring) under
    the local-search plan annealed over its contraction tree and the choice of its 10 sliced bonds
    (qxgen/plans/grid6x6_d14_s10_open6_sa.json): 1024 slices of other sub-networks, whose sum is the
    same amplitude vector (Eq. 2), with most steps independent of the slice."""
    from .plan import sliceable_bonds
    base = large()
    order, sliced, peak, flops, executed, d = _load_stored_plan("grid6x6_d14_s10_open6_sa.json", base.circuit,
                                                                base.open_mask, len(base.bitstrings))
    legs, _, open_edges = network_legs(base.n_qubits, [g.qubits for g in base.circuit.gates], base.open_mask)
    ok = set(sliceable_bonds(legs, base.n_qubits - len(open_edges), open_edges))
    if len(sliced) != len(base.sliced) or len(set(sliced)) != len(sliced) or not set(sliced) <= ok:
        raise ValueError("stored plan does not slice 10 distinct sliceable bonds")
    return Workload("grid6x6_d14_s10_open6_sa", base.circuit, base.open_mask, order, sliced, base.bitstrings, peak,
                    flops, {"plan": "local-search plan annealed over its tree and its sliced bonds (stored)",
                            "executed_flops": executed, "made_by": d["made_by"]})


@functools.lru_cache(maxsize=None)
def large():
    cseed = 3001
    circ = random_grid_circuit(6, 6, 14, cseed)
    om = np.zeros(36, np.uint8)
    om[30:] = 1
    bits = random_bitstrings(36, 1, cseed + 500000)
    return _workload("grid6x6_d14_s10_open6", circ, om, 10, cseed, bits, trials=64, peak_rank=28)


def batched_specs(count=256):
    """Per-circuit (n, depth, n_slice, n_bits) draws of the batched workload."""
    rng = SplitMix64(4000)
    specs = []
    for j in range(count):
        n = 16 + rng.randint(13)
        depth = 8 + rng.randint(9)
        s = rng.randint(9)
        nb = 1 + rng.randint(64)
        specs.append((n, depth, s, nb))
    return specs


@functools.lru_cache(maxsize=None)
def batched_circuit_greedy(j):
    """Circuit j of the batched workload under a seeded greedy plan with its drawn S sliced bonds (the
    starting point of its stored plan)."""
    n, depth, s, nb = batched_specs()[j]
    cseed = 4000 + j
    rows, cols = near_square_shape(n)
    circ = random_grid_circuit(rows, cols, depth, cseed, n=n)
    bits = random_bitstrings(n, nb, cseed + 500000)
    return _workload(f"batched{j}_n{n}_d{depth}_s{s}", circ, np.zeros(n, np.uint8), s, cseed, bits,
                     trials=1, meta={"n": n, "depth": depth, "j": j})


@functools.lru_cache(maxsize=None)
def _batched_plans():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans", "batched_uneven.json")
    with open(path) as f:
        return json.load(f)["plans"]


@functools.lru_cache(maxsize=None)
def _batched_annealed_plans():
    """The annealed plans of the batched workload's heaviest circuits, by circuit index (may be empty)."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans", "batched_annealed.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return {d["j"]: d for d in json.load(f)["plans"]}


@functools.lru_cache(maxsize=None)
def batched_circuit(j, annealed=True):
    """Circuit j of the batched workload under its stored plan, checked against the circuit and its
    recorded cost: qxgen/plans/batched_annealed.json for the heaviest circuits (their plans annealed over
    the tree and the choice of their sliced bonds, the drawn number kept), else
    qxgen/plans/batched_uneven.json (level-aware candidates + local search on the time estimate; both
    written by qxgen.make_plans).  annealed=False gives the latter for every circuit."""
    g = batched_circuit_greedy(j)
    d = _batched_annealed_plans().get(j) if annealed else None
    d = d or _batched_plans()[j]
    n, depth, s, nb = batched_specs()[j]
    if d["j"] != j or d["circuit_sha256"] != circuit_digest(g.circuit) or d["n_bits"] != nb or len(d["sliced"]) != s:
        raise ValueError(f"stored plan {j} was made for another circuit")
    if len(set(d["sliced"])) != s:
        raise ValueError(f"stored plan {j} repeats a sliced bond")
    order = [tuple(p) for p in d["order"]]
    legs, _, open_edges = network_legs(n, [x.qubits for x in g.circuit.gates], g.open_mask)
    peak, flops = plan_cost(legs, order, d["sliced"])
    if executed_cost(legs, order, d["sliced"], n - len(open_edges), nb) != d["executed_flops"] or peak > d["max_peak"]:
        raise ValueError(f"stored plan {j} does not match its recorded cost")
    return Workload(g.name, g.circuit, g.open_mask, order, list(d["sliced"]), g.bitstrings, peak, flops,
                    {"n": n, "depth": depth, "j": j, "executed_flops": d["executed_flops"],
                     "estimated_s": d["estimated_s"]})


def batched_members(count=256):
    """All circuits of the batched workload under their stored plans."""
    return [batched_circuit(j) for j in range(count)]


def serving_specs(count=32):
    """Per-circuit (n, depth) draws of the serving workload."""
    rng = SplitMix64(5000)
    return [(20 + rng.randint(21), 10 + rng.randint(7)) for _ in range(count)]


def serving_base(j):
    """(name, circuit, bitstring) of resident circuit j of the serving workload (no plan)."""
    n, depth = serving_specs()[j]
    cseed = 5000 + j
    rows, cols = near_square_shape(n)
    circ = random_grid_circuit(rows, cols, depth, cseed, n=n)
    return f"serving{j}_n{n}_d{depth}", circ, random_bitstrings(n, 1, cseed + 500000)


@functools.lru_cache(maxsize=None)
def serving_circuit_greedy(j, peak_rank=30):
    """Resident circuit j of the serving workload under a seeded greedy plan, sliced until its peak fits
    2^peak_rank entries."""
    name, circ, bits = serving_base(j)
    n, depth = serving_specs()[j]
    return _workload(name, circ, np.zeros(n, np.uint8), 0, 5000 + j, bits, trials=1,
                     peak_rank=peak_rank, meta={"n": n, "depth": depth, "j": j})


@functools.lru_cache(maxsize=None)
def _serving_plans():
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans", "serving.json")
    with open(path) as f:
        return json.load(f)["plans"]


@functools.lru_cache(maxsize=None)
def serving_circuit(j):
    """Resident circuit j of the serving workload under its stored plan (qxgen/plans/serving.json,
    written by qxgen.make_plans), checked against the circuit and its recorded cost."""
    name, circ, bits = serving_base(j)
    d = _serving_plans()[j]
    n, depth = serving_specs()[j]
    om = np.zeros(n, np.uint8)
    if d["j"] != j or d["circuit_sha256"] != circuit_digest(circ):
        raise ValueError(f"stored serving plan {j} was made for another circuit")
    order = [tuple(p) for p in d["order"]]
    legs, _, open_edges = network_legs(n, [x.qubits for x in circ.gates], om)
    peak, flops = plan_cost(legs, order, d["sliced"])
    if executed_cost(legs, order, d["sliced"], n - len(open_edges), d["n_bits"]) != d["executed_flops"] or \
            peak > d["max_peak"]:
        raise ValueError(f"stored serving plan {j} does not match its recorded cost")
    return Workload(name, circ, om, order, list(d["sliced"]), bits, peak, flops,
                    {"n": n, "depth": depth, "j": j, "executed_flops_256": d["executed_flops"],
                     "estimated_s_256": d["estimated_s"], "estimated_s_1": d["estimated_s_1bit"]})
