"""Write the stored plans of qxgen/plans/ (plans are inputs; the paper keeps them in files).

    python -m qxgen.make_plans [checkpoint] [large]

grid4x5_d12_s6_checkpoint.json: the 20-qubit sliced circuit (4x5 grid, depth
12, six sliced bonds, 256 bitstrings) under the level-aware plan improved by
local search (20000 seeded tree rotations), which about 25 s of host time
finds; the workload loads it instead of searching again.

grid6x6_d14_s10_open6_ls.json: the 36-qubit large workload (6x6 grid, depth
14, qubits 30..35 open, 10 sliced bonds) under its seeded plan improved by
local search (150000 rotations, about 6 minutes of host time): 2.4e13 instead
of 1.0e15 executed flops per call, the same sliced bonds, peak 2^22 entries.
"""
import json
import os

from . import workloads as W
from .plan import local_search_plan, network_legs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "plans")


def checkpoint_plan():
    base = W.sliced_level_aware()
    circ = base.circuit
    legs, _, open_edges = network_legs(circ.n_qubits, [g.qubits for g in circ.gates], base.open_mask)
    n_out = circ.n_qubits - len(open_edges)
    order, executed, accepted = local_search_plan(legs, base.order, base.sliced, n_out, len(base.bitstrings),
                                                  max_peak=14, iters=20000, seed=11)
    return {"circuit_sha256": W.circuit_digest(circ), "order": [list(p) for p in order],
            "sliced": [int(e) for e in base.sliced], "executed_flops": int(executed),
            "n_bits": int(len(base.bitstrings)), "max_peak": 14,
            "made_by": "level_aware_plan (40 trials per setting, seed 702001) + local_search_plan "
                       "(20000 rotations, seed 11)"}


def large_plan(iters=150000, seed=13):
    """The large workload's seeded plan improved by local search; the sliced bonds stay those of the
    seeded plan, so its slices are the same sub-networks (Eq. 2) in another contraction order."""
    base = W.large()
    circ = base.circuit
    legs, _, open_edges = network_legs(circ.n_qubits, [g.qubits for g in circ.gates], base.open_mask)
    n_out = circ.n_qubits - len(open_edges)
    order, executed, accepted = local_search_plan(legs, base.order, base.sliced, n_out, len(base.bitstrings),
                                                  max_peak=28, iters=iters, seed=seed)
    return {"circuit_sha256": W.circuit_digest(circ), "order": [list(p) for p in order],
            "sliced": [int(e) for e in base.sliced], "executed_flops": int(executed),
            "n_bits": int(len(base.bitstrings)), "max_peak": 28,
            "made_by": f"randomized_greedy (64 trials per setting, seed 703001) + tree trimming + "
                       f"local_search_plan ({iters} rotations, seed {seed})"}


def _write(name, d):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(d, f)
    print(path, d["executed_flops"])


if __name__ == "__main__":
    import sys
    os.makedirs(HERE, exist_ok=True)
    which = sys.argv[1:] or ["checkpoint", "large"]
    if "checkpoint" in which:
        _write("grid4x5_d12_s6_checkpoint.json", checkpoint_plan())
    if "large" in which:
        _write("grid6x6_d14_s10_open6_ls.json", large_plan())
