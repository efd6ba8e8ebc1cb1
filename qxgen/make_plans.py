"""Write the stored plans of qxgen/plans/ (plans are inputs; the paper keeps them in files).

    python -m qxgen.make_plans [checkpoint] [large] [annealed] [batched] [batched-annealed] [serving]

grid4x5_d12_s6_checkpoint.json: the 20-qubit sliced circuit (4x5 grid, depth
12, six sliced bonds, 256 bitstrings) under the level-aware plan improved by
local search (20000 seeded tree rotations), which about 25 s of host time
finds; the workload loads it instead of searching again.

grid6x6_d14_s10_open6_ls.json: the 36-qubit large workload (6x6 grid, depth
14, qubits 30..35 open, 10 sliced bonds) under its seeded plan improved by
local search: 150000 rotations on executed flops, 20000 on the step-level
time estimate, 20000 on the compiled launch-list time (about 15 minutes of
host time).  The result executes 3.1e13 instead of 1.0e15 flops per call,
with the same sliced bonds and a peak of 2^22 entries.

grid6x6_d14_s10_open6_sa.json: the same workload under the local-search plan
annealed on the compiled launch-list time over its contraction tree and its
choice of 10 sliced bonds (80000 iterations, about 40 minutes of host time).

batched_uneven.json: the 256 circuits of the batched workload, each under
its level-aware plan improved by local search on the time estimate (about
half an hour of host time on 7 processes).

batched_annealed.json: the heaviest of those circuits under their stored
plans annealed on the compiled launch-list time over the tree and the
choice of their sliced bonds (the drawn number kept); the workload uses
these entries in place of batched_uneven.json's.

serving.json: the 32 resident circuits of the serving workload, each under
the seeded greedy candidate that, sliced until its intermediates fit 2^30
entries, has the smallest time estimate for 256 bitstrings, improved by
local search on that estimate.
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


def large_plan(iters=150000, seed=12, iters_t=20000, seed_t=51, iters_c=20000, seed_c=52):
    """The large workload's seeded plan improved by local search in three passes: on executed flops, on
    the step-level time estimate (executed_time: memory traffic counts too), and on the time of the
    launch list the library compiles for it (qxgen.compiled_cost: kernel families, permutes, shared
    operands).  The sliced bonds stay those of the seeded plan, so its slices are the same sub-networks
    (Eq. 2) in another contraction order."""
    from .compiled_cost import CompiledTime
    from .plan import executed_cost
    base = W.large()
    circ = base.circuit
    legs, _, open_edges = network_legs(circ.n_qubits, [g.qubits for g in circ.gates], base.open_mask)
    n_out = circ.n_qubits - len(open_edges)
    nb = len(base.bitstrings)
    order, _, _ = local_search_plan(legs, base.order, base.sliced, n_out, nb, max_peak=28, iters=iters, seed=seed)
    order, _, _ = local_search_plan(legs, order, base.sliced, n_out, nb, max_peak=28, iters=iters_t, seed=seed_t,
                                    objective="time")
    obj = CompiledTime(circ.n_qubits, base.gates, base.open_mask, precision=1)
    order, t, _ = local_search_plan(legs, order, base.sliced, n_out, nb, max_peak=28, iters=iters_c, seed=seed_c,
                                    objective=obj)
    obj.close()
    return {"circuit_sha256": W.circuit_digest(circ), "order": [list(p) for p in order],
            "sliced": [int(e) for e in base.sliced], "executed_flops": int(executed_cost(legs, order, base.sliced,
                                                                                          n_out, nb)),
            "estimated_s": t, "n_bits": int(nb), "max_peak": 28,
            "made_by": f"randomized_greedy (64 trials per setting, seed 703001) + tree trimming + "
                       f"local_search_plan ({iters} rotations, seed {seed}, executed flops) + "
                       f"local_search_plan ({iters_t} rotations, seed {seed_t}, time estimate) + "
                       f"local_search_plan ({iters_c} rotations, seed {seed_c}, compiled launch-list time)"}


ANNEALED_MAX_PEAK = 24  # 2^24 complex64 entries = 128 MiB per intermediate


def large_annealed_plan(seed=203, iters=80000, p_swap=0.15, t_start=3e-3, t_end=1e-5):
    """The large workload's local-search plan (the stored one) annealed on the compiled launch-list
    time (qxgen.compiled_cost) over its contraction tree and its choice of 10 sliced bonds
    (qxgen.plan.anneal_plan).  Tree trimming slices the bonds that shrink the largest intermediate;
    once the steps no sliced bond reaches run once per call, the cheaper choice slices bonds that few
    steps depend on.  Seeds 201..207 were run with these settings (p_swap 0.3, 0.15 or 0.5); the
    stored plan is the cheapest result."""
    from .compiled_cost import CompiledTime
    from .plan import anneal_plan, executed_cost, plan_cost, sliceable_bonds
    base = W.large_local_search()
    circ = base.circuit
    legs, _, open_edges = network_legs(circ.n_qubits, [g.qubits for g in circ.gates], base.open_mask)
    n_out = circ.n_qubits - len(open_edges)
    nb = len(base.bitstrings)
    obj = CompiledTime(circ.n_qubits, base.gates, base.open_mask, precision=1)
    order, sliced, t, _ = anneal_plan(legs, base.order, base.sliced, n_out, nb, ANNEALED_MAX_PEAK, iters, seed, obj,
                                      sliceable_bonds(legs, n_out, open_edges), p_swap, t_start, t_end)
    obj.close()
    return {"circuit_sha256": W.circuit_digest(circ), "order": [list(p) for p in order],
            "sliced": [int(e) for e in sliced], "executed_flops": int(executed_cost(legs, order, sliced, n_out, nb)),
            "estimated_s": t, "n_bits": int(nb), "max_peak": ANNEALED_MAX_PEAK,
            "peak": plan_cost(legs, order, sliced)[0],
            "made_by": f"the stored local-search plan + anneal_plan ({iters} iterations, seed {seed}, swap "
                       f"probability {p_swap}, temperature {t_start} -> {t_end} of the starting cost, compiled "
                       f"launch-list time, peak 2^{ANNEALED_MAX_PEAK})"}


BATCHED_MAX_PEAK = 28


def batched_plan(j, trials=20, iters=20000):
    """Circuit j of the batched uneven workload: its drawn number of sliced bonds S, the seeded greedy
    candidates ranked by executed flops (level_aware_plan), then local search on the time estimate
    (executed_time), every intermediate within 2^28 entries."""
    from .plan import executed_cost, executed_time, level_aware_plan, plan_cost
    n, depth, S, nb = W.batched_specs()[j]
    w = W.batched_circuit_greedy(j)
    circ = w.circuit
    legs, _, open_edges = network_legs(n, [g.qubits for g in circ.gates], w.open_mask)
    n_out = n - len(open_edges)
    no_slice = list(open_edges) + [legs[t][0] for t in range(len(legs) - n_out, len(legs))]
    order, sliced, _, _ = level_aware_plan(legs, trials, 4000 + j + 700000, S, no_slice, n_out, nb,
                                           max_peak=BATCHED_MAX_PEAK)
    order, t, _ = local_search_plan(legs, order, sliced, n_out, nb, BATCHED_MAX_PEAK, iters, j, objective="time")
    return {"j": j, "circuit_sha256": W.circuit_digest(circ), "order": [list(p) for p in order],
            "sliced": [int(e) for e in sliced], "n_bits": nb, "max_peak": BATCHED_MAX_PEAK,
            "peak": plan_cost(legs, order, sliced)[0], "executed_flops": int(executed_cost(legs, order, sliced, n_out, nb)),
            "estimated_s": t}


def batched_annealed_plan(j, seed, iters, t_start, start="stored"):
    """Circuit j of the batched workload: a starting order -- its stored plan (batched_uneven.json), or
    with start="sweep" the state-vector-like sweep_order with the stored sliced bonds -- annealed on the
    compiled launch-list time of a 3xTF32 call (qxgen.compiled_cost) over its contraction tree and, when
    it slices bonds, its choice of them (swap probability 0.15; the drawn number kept), every
    intermediate within 2^28 entries."""
    from .compiled_cost import CompiledTime
    from .plan import anneal_plan, executed_cost, plan_cost, sliceable_bonds, sweep_order
    w = W.batched_circuit(j, annealed=False)
    circ = w.circuit
    gq = [g.qubits for g in circ.gates]
    legs, _, open_edges = network_legs(circ.n_qubits, gq, w.open_mask)
    n_out = circ.n_qubits - len(open_edges)
    nb = len(w.bitstrings)
    order0 = sweep_order(legs, circ.n_qubits, n_out, gq) if start == "sweep" else w.order
    obj = CompiledTime(circ.n_qubits, w.gates, w.open_mask, precision=1)
    stored = obj(legs, w.order, w.sliced, n_out, nb)
    p_swap = 0.15 if w.sliced else 0.0
    order, sliced, t, _ = anneal_plan(legs, order0, w.sliced, n_out, nb, BATCHED_MAX_PEAK, iters, seed, obj,
                                      sliceable_bonds(legs, n_out, open_edges), p_swap, t_start, 1e-5)
    obj.close()
    return {"j": j, "circuit_sha256": W.circuit_digest(circ), "order": [list(p) for p in order],
            "sliced": [int(e) for e in sliced], "n_bits": nb, "max_peak": BATCHED_MAX_PEAK,
            "peak": plan_cost(legs, order, sliced)[0], "executed_flops": int(executed_cost(legs, order, sliced, n_out, nb)),
            "estimated_s": t, "stored_estimated_s": stored,
            "made_by": f"{'sweep_order' if start == 'sweep' else 'the stored plan'} + anneal_plan ({iters} iterations, "
                       f"seed {seed}, swap probability {p_swap}, temperature {t_start} -> 1e-05 of the starting "
                       f"cost, compiled launch-list time)"}


# (circuit, seed, iterations, starting temperature, start) of the batched workload's annealed plans:
# its heaviest circuits by estimated time; the rest keep their batched_uneven.json plans
BATCHED_ANNEALED = ((39, 1, 20000, 0.003, "sweep"), (71, 1, 20000, 0.003, "sweep"), (72, 1072, 20000, 0.01, "stored"),
                    (73, 73, 20000, 0.003, "stored"), (91, 1, 20000, 0.003, "sweep"), (94, 1, 20000, 0.003, "sweep"),
                    (102, 1, 20000, 0.003, "sweep"), (120, 120, 30000, 0.003, "stored"),
                    (125, 1125, 20000, 0.01, "stored"), (137, 1, 20000, 0.003, "sweep"),
                    (146, 146, 30000, 0.003, "stored"), (149, 1, 20000, 0.003, "sweep"),
                    (162, 1, 20000, 0.003, "sweep"), (170, 2, 20000, 0.003, "sweep"), (181, 2, 20000, 0.003, "sweep"),
                    (223, 1, 20000, 0.003, "sweep"), (243, 1243, 60000, 0.01, "stored"))


def _annealed_entry(args):
    return batched_annealed_plan(*args)


def batched_annealed_plans(workers=7):
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        plans = pool.map(_annealed_entry, BATCHED_ANNEALED, chunksize=1)
    return {"made_by": "the heaviest circuits' stored plans annealed on the compiled launch-list time "
                       "(batched_annealed_plan); an entry replaces the circuit's plan in batched_uneven.json",
            "plans": plans}


def batched_plans(workers=7):
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        plans = pool.map(batched_plan, range(256), chunksize=1)
    return {"made_by": "per circuit: level_aware_plan (20 trials per setting, seed 704000 + j) + local_search_plan "
                       "(20000 rotations, seed j, objective time), max peak 2^28",
            "plans": plans}


SERVING_MAX_PEAK = 30  # 2^30 complex64 entries = 8 GB per intermediate
SERVING_PLAN_BITS = 256  # bitstrings per call the serving plans are ranked for


def serving_plan(j, trials=10, iters=5000):
    """Resident circuit j of the serving workload: seeded greedy candidates, each sliced by tree trimming
    until every intermediate fits 2^30 entries, ranked by the time estimate of a call of 256 bitstrings
    (fitted_plan), then local search on that estimate."""
    from .plan import executed_cost, executed_time, fitted_plan, plan_cost
    import numpy as np
    _, circ, _ = W.serving_base(j)
    n = circ.n_qubits
    legs, _, open_edges = network_legs(n, [g.qubits for g in circ.gates], np.zeros(n, np.uint8))
    n_out = n - len(open_edges)
    no_slice = list(open_edges) + [legs[t][0] for t in range(len(legs) - n_out, len(legs))]
    nb = SERVING_PLAN_BITS
    order, sliced, _ = fitted_plan(legs, trials, 5000 + j + 700000, no_slice, n_out, nb, SERVING_MAX_PEAK)
    order, t, _ = local_search_plan(legs, order, sliced, n_out, nb, SERVING_MAX_PEAK, iters, j, objective="time")
    return {"j": j, "circuit_sha256": W.circuit_digest(circ), "order": [list(p) for p in order],
            "sliced": [int(e) for e in sliced], "n_bits": nb, "max_peak": SERVING_MAX_PEAK,
            "peak": plan_cost(legs, order, sliced)[0],
            "executed_flops": int(executed_cost(legs, order, sliced, n_out, nb)), "estimated_s": t,
            "estimated_s_1bit": executed_time(legs, order, sliced, n_out, 1)}


def serving_plans(workers=3):
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        plans = pool.map(serving_plan, range(32), chunksize=1)
    return {"made_by": "per circuit: fitted_plan (10 trials per setting, seed 705000 + j, sliced to 2^30 entries, "
                       "ranked for 256 bitstrings), then local_search_plan (5000 rotations, seed j, objective time)",
            "plans": plans}


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
    if "annealed" in which:
        _write("grid6x6_d14_s10_open6_sa.json", large_annealed_plan())
    if "serving" in which:
        d = serving_plans()
        path = os.path.join(HERE, "serving.json")
        with open(path, "w") as f:
            json.dump(d, f)
        print(path, [round(p["estimated_s"], 3) for p in d["plans"]])
    if "batched-annealed" in which:
        d = batched_annealed_plans()
        path = os.path.join(HERE, "batched_annealed.json")
        with open(path, "w") as f:
            json.dump(d, f)
        print(path, [(p["j"], round(p["stored_estimated_s"], 3), round(p["estimated_s"], 3)) for p in d["plans"]])
    if "batched" in which:
        d = batched_plans()
        path = os.path.join(HERE, "batched_uneven.json")
        with open(path, "w") as f:
            json.dump(d, f)
        print(path, sum(p["estimated_s"] for p in d["plans"]))
