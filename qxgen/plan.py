"""Contraction plans for circuit tensor networks (input generation only).

A plan is the pair (order, sliced): a pairwise contraction order in SSA form
and a list of bond indices to slice.  The paper treats finding both as the
high-level challenge solved before any amplitude is computed (Sec. III-A);
QuantEx uses FlowCutter tree decompositions for the order and the greedy
"tree trimming" rule of Schutski et al. for the sliced bonds.  This module
supplies stand-ins that produce valid plans for the synthetic workloads:

* ``greedy_order``: repeatedly contract the pair of tensors sharing a bond
  that minimises size(out) - size(A) - size(B), ties to the lowest SSA ids;
  ``randomized_greedy`` perturbs that cost with seeded Gumbel noise and keeps
  the best of several trials (a common way to improve on plain greedy).
* ``tree_trim_slices``: the greedy slicing rule of Sec. III-A: slice a bond
  that shrinks the largest intermediate; among those prefer the one in the
  most largest intermediates, then the one in the most intermediates, then
  the one saving the most total memory, then a seeded random choice.
* ``level_aware_plan`` / ``local_search_plan`` / ``anneal_plan``: plans
  ranked by what a call executes when steps run at their dependence level
  (``executed_cost``, ``executed_time`` or the library's compiled launch
  list), improved by seeded tree rotations and, in ``anneal_plan``, swaps of
  sliced bonds under a cooling Metropolis rule; ``sweep_order`` is a
  state-vector-like starting order whose steps below the final layer reach
  no output bit.

Only index bookkeeping lives here (which bond sits on which tensor); no
tensor values are touched.  The network labelling below is the canonical
one of the C-ABI (tensor ids: inputs, gates, outputs of closed qubits; bond
ids: input wires 0..n-1, then each gate's output legs in creation order).
"""
from __future__ import annotations

import heapq
import math

from .circuits import SplitMix64


def network_legs(n_qubits: int, gate_qubits, open_mask=None):
    """Canonical tensor legs.

    Returns (legs, n_edges, open_edges): legs[t] is the list of bond ids on
    tensor t in its storage order.  Inputs have [wire]; a one-qubit gate has
    [out, in]; a two-qubit gate has [out0, out1, in0, in1]; outputs [wire].
    """
    if open_mask is None:
        open_mask = [0] * n_qubits
    wire = list(range(n_qubits))
    legs = [[q] for q in range(n_qubits)]
    ne = n_qubits
    for qs in gate_qubits:
        outs = []
        for q in qs:
            outs.append(ne)
            ne += 1
        legs.append(outs + [wire[q] for q in qs])
        for q, e in zip(qs, outs):
            wire[q] = e
    open_edges = []
    for q in range(n_qubits):
        if open_mask[q]:
            open_edges.append(wire[q])
        else:
            legs.append([wire[q]])
    return legs, ne, open_edges


def _greedy(legs, noise_rng=None, temperature=0.0, alpha=1.0):
    n0 = len(legs)
    sets = {i: frozenset(l) for i, l in enumerate(legs)}
    owner = {}
    for i, s in sets.items():
        for e in s:
            owner.setdefault(e, set()).add(i)

    def cost(a, b):
        sa, sb = sets[a], sets[b]
        c = float((1 << len(sa ^ sb)) - alpha * ((1 << len(sa)) + (1 << len(sb))))
        if noise_rng is not None and temperature > 0:
            u = max(noise_rng.uniform(), 1e-300)
            # Gumbel-perturbed log-size cost keeps the scale of large tensors comparable
            c = math.copysign(math.log2(1 + abs(c)), c) - temperature * math.log(-math.log(u) + 1e-300)
        return c

    heap = []

    def push_pairs(i):
        nb = set()
        for e in sets[i]:
            nb |= owner[e]
        nb.discard(i)
        for j in nb:
            a, b = (i, j) if i < j else (j, i)
            heapq.heappush(heap, (cost(a, b), a, b))

    for i in list(sets):
        push_pairs(i)
    order = []
    nxt = n0
    while len(sets) > 1:
        pair = None
        while heap:
            c, a, b = heapq.heappop(heap)
            if a in sets and b in sets:
                pair = (a, b)
                break
        if pair is None:  # disconnected components: outer product of the two lowest ids
            ids = sorted(sets)
            pair = (ids[0], ids[1])
        a, b = pair
        out = sets[a] ^ sets[b]
        for e in sets[a] | sets[b]:
            owner[e].discard(a)
            owner[e].discard(b)
        del sets[a], sets[b]
        sets[nxt] = out
        for e in out:
            owner[e].add(nxt)
        order.append((a, b))
        push_pairs(nxt)
        nxt += 1
    return order


def greedy_order(legs):
    """Deterministic greedy SSA order (see module docstring)."""
    return _greedy(legs)


def intermediates(legs, order):
    """Bond sets of every tensor created by the plan, in step order."""
    sets = [frozenset(l) for l in legs]
    out = []
    for a, b in order:
        s = sets[a] ^ sets[b]
        sets.append(s)
        out.append(s)
    return out


def plan_cost(legs, order, sliced=()):
    """(max rank, total flops per slice (8 M K N convention), total entries written) of a plan."""
    sl = frozenset(sliced)
    sets = [frozenset(l) - sl for l in legs]
    max_rank = 0
    flops = 0
    for a, b in order:
        sa, sb = sets[a], sets[b]
        shared = sa & sb
        out = sa ^ sb
        m, k, n = len(sa - shared), len(shared), len(sb - shared)
        flops += 8 * (1 << (m + k + n))
        max_rank = max(max_rank, len(out))
        sets.append(out)
    return max_rank, flops


def tree_trim_slices(legs, order, n_slice, seed=0, open_edges=()):
    """Greedy tree-trimming choice of n_slice bonds to slice (Sec. III-A).

    Bonds listed in open_edges are never chosen (pass every qubit's final
    wire: open ones are not bonds and closed ones carry the bitstring).
    """
    rng = SplitMix64(seed)
    inter = intermediates(legs, order)
    open_set = frozenset(open_edges)
    sliced = []
    for _ in range(n_slice):
        sl = frozenset(sliced)
        ranks = [len(s - sl) for s in inter]
        # the largest intermediates that still hold a sliceable bond
        cands = set()
        for rmax in sorted(set(ranks), reverse=True):
            largest = [s - sl for s, r in zip(inter, ranks) if r == rmax]
            for s in largest:
                cands |= s
            cands -= open_set
            if cands:
                break
        if not cands:
            raise ValueError("no bond left to slice")
        best = None
        for e in sorted(cands):
            k1 = sum(1 for s in largest if e in s)
            k2 = sum(1 for s in inter if e in s and e not in sl)
            k3 = sum(1 << (r - 1) for s, r in zip(inter, ranks) if e in s)
            key = (k1, k2, k3, rng.next_u64())
            if best is None or key > best[0]:
                best = (key, e)
        sliced.append(best[1])
    return sliced


def randomized_greedy(legs, trials, seed, n_slice=0, open_edges=(), settings=((1.0, 0.6), (0.75, 0.3),
                      (0.75, 0.6), (0.5, 0.6), (0.25, 0.3)), keep=6):
    """Best plan over seeded Gumbel-perturbed greedy orders.

    Each (alpha, temperature) setting runs `trials` orders with the cost
    size(out) - alpha (size(A) + size(B)); the `keep` cheapest orders by
    unsliced flops are then sliced by tree trimming and the plan with the
    fewest flops after slicing (then the smallest peak) wins.  The
    deterministic greedy order is always a candidate.
    """
    rng = SplitMix64(seed)
    cands = [(plan_cost(legs, o)[1], 0, o) for o in [_greedy(legs)]]
    k = 1
    for alpha, temp in settings:
        for _ in range(trials):
            o = _greedy(legs, rng, temp, alpha)
            cands.append((plan_cost(legs, o)[1], k, o))
            k += 1
    cands.sort(key=lambda c: (c[0], c[1]))
    best = None
    for flops0, k, order in cands[:keep]:
        sliced = tree_trim_slices(legs, order, n_slice, seed + k, open_edges) if n_slice else []
        peak, flops = plan_cost(legs, order, sliced)
        key = (flops, peak, k)
        if best is None or key < best[0]:
            best = (key, order, sliced)
    return best[1], best[2]


def executed_cost(legs, order, sliced, n_outputs, n_bits):
    """Flops one contraction call executes when steps run at their dependence level.

    A step that no sliced bond and no output bit reaches runs once, one that a
    sliced bond reaches but no output bit runs once per slice, the others once
    per (slice, bitstring) pair (n_bits bitstrings per call); a step is reached
    by a fixed bond when any leaf below it touches that bond.  The last
    n_outputs tensors are the closed outputs <x_q|: their bonds are fixed, and
    absorbing one is a relabelling with no flops.  A step costs 8 M K N over
    its unfixed bonds.
    """
    sl = frozenset(sliced)
    first_out = len(legs) - n_outputs
    out_wires = frozenset(e for t in range(first_out, len(legs)) for e in legs[t])
    fixed = sl | out_wires
    sets = [frozenset(l) for l in legs]
    # a fixed bond is read as an address offset on every leaf it touches, so a leaf on a closed
    # output wire depends on the bitstring, one on a sliced bond on the slice
    by_slice = [bool(sl & sets[t]) for t in range(len(legs))]
    by_bits = [bool(out_wires & sets[t]) for t in range(len(legs))]
    n_slices = 1 << len(sl)
    total = 0
    for a, b in order:
        sa, sb = sets[a] - fixed, sets[b] - fixed
        shared = sa & sb
        closing = (a >= first_out and a < len(legs)) or (b >= first_out and b < len(legs))
        flops = 0 if closing else 8 * (1 << (len(sa - shared) + len(shared) + len(sb - shared)))
        s_dep, b_dep = by_slice[a] or by_slice[b], by_bits[a] or by_bits[b]
        total += flops * (n_slices * n_bits if b_dep else n_slices if s_dep else 1)
        sets.append(sets[a] ^ sets[b])
        by_slice.append(s_dep)
        by_bits.append(b_dep)
    return total


# Rates of one GB300 for executed_time, in the units of the 8 M K N convention and bytes, from the
# kernels' measured throughput on the 36-qubit sliced workload: tensor-core products in 3xTF32 (about
# 170 complex TFLOP/s), the SIMT complex64 GEMM, the gather kernels' FP32 arithmetic, and the HBM
# bandwidth the memory-bound kernels reach (about 4.7 TB/s); plus a fixed cost per launch.
GB300_RATES = {"tc": 170e12, "gemm": 35e12, "gather": 20e12, "hbm": 4.7e12, "launch": 4e-6}


def step_kind(m, k, n, small_entries, tensor_cores=True):
    """The kernel family the library's plan compiler picks for a step with m, k, n free / shared /
    free bits (m >= n): 'gather' when one operand has at most 2^10 entries, k <= 5 and that operand
    has at most 5 free bits (and the step is not a GEMM with all three >= 5), 'tc' for the tensor-core
    shapes of the 3xTF32 form, else 'gemm'."""
    big_gemm = k >= 5 and m >= 5 and n >= 5
    if small_entries <= 10 and k <= 5 and n <= 5 and not big_gemm:
        return "gather"
    if tensor_cores and ((m >= 7 and n >= 5 and k >= 4 and (m <= 8 or n <= 8)) or (m >= 7 and n >= 6 and k >= 5)):
        return "tc"
    return "gemm"


def executed_time(legs, order, sliced, n_outputs, n_bits, rates=GB300_RATES, tensor_cores=True):
    """Estimated seconds of one contraction call on one GPU, steps at their dependence level.

    Each step is one launch over its items (1, the slices, or the (slice, bitstring) pairs); it takes
    the longer of its flops at its kernel family's rate (step_kind) and its bytes at the HBM rate,
    8 (|A| + |B| + |C|) per item with an operand of a lower level (shared by the items) read once,
    plus the launch cost.  A roofline estimate: it ignores permutes and overlap between launches, and
    serves to rank plans, where executed flops alone favour huge tensors contracted over few bonds
    (cheap in flops, bound by memory traffic)."""
    sl = frozenset(sliced)
    first_out = len(legs) - n_outputs
    out_wires = frozenset(e for t in range(first_out, len(legs)) for e in legs[t])
    fixed = sl | out_wires
    sets = [frozenset(l) for l in legs]
    lev = [2 if out_wires & sets[t] else 1 if sl & sets[t] else 0 for t in range(len(legs))]
    n_slices = 1 << len(sl)
    mult = (1, n_slices, n_slices * n_bits)
    total = 0.0
    for a, b in order:
        sa, sb = sets[a] - fixed, sets[b] - fixed
        la = lev[a]
        lb = lev[b]
        lc = max(la, lb)
        closing = first_out <= a < len(legs) or first_out <= b < len(legs)
        sets.append(sets[a] ^ sets[b])
        lev.append(lc)
        if closing:
            continue
        shared = sa & sb
        m, k, n = len(sa - shared), len(shared), len(sb - shared)
        ea, eb = len(sa), len(sb)
        if m < n:
            m, n = n, m
        kind = step_kind(m, k, n, min(ea, eb), tensor_cores)
        items = mult[lc]
        flops = 8.0 * 2.0 ** (m + k + n) * items
        nbytes = 8.0 * (2.0 ** (m + n) * items + 2.0 ** ea * (items if la == lc else 1)
                        + 2.0 ** eb * (items if lb == lc else 1))
        total += max(flops / rates[kind], nbytes / rates["hbm"]) + rates["launch"]
    return total


def level_aware_plan(legs, trials, seed, n_slice, open_edges, n_outputs, n_bits, max_peak=None,
                     settings=((1.0, 0.6), (0.75, 0.3), (0.75, 0.6), (0.5, 0.6), (0.25, 0.3), (1.0, 1.0),
                               (1.0, 0.2)), max_pair_peak=None):
    """Seeded greedy orders, each sliced by tree trimming, ranked by executed_cost.

    Same candidates as randomized_greedy (Gumbel-perturbed greedy orders under
    several (alpha, temperature) settings, plus the deterministic greedy
    order), but every one is sliced and the plan that executes the fewest
    flops per call of n_bits bitstrings wins (ties: smaller peak, earlier
    candidate), among those whose largest intermediate has at most max_peak
    legs.  Returns (order, sliced, executed flops, peak rank).
    """
    rng = SplitMix64(seed)
    orders = [_greedy(legs)]
    for alpha, temp in settings:
        for _ in range(trials):
            orders.append(_greedy(legs, rng, temp, alpha))
    best = None
    for k, order in enumerate(orders):
        sliced = tree_trim_slices(legs, order, n_slice, seed + k, open_edges) if n_slice else []
        peak, _ = plan_cost(legs, order, sliced)
        if max_peak is not None and peak > max_peak:
            continue
        if max_pair_peak is not None and pair_peak(legs, order, sliced, n_outputs) > max_pair_peak:
            continue
        ex = executed_cost(legs, order, sliced, n_outputs, n_bits)
        key = (ex, peak, k)
        if best is None or key < best[0]:
            best = (key, order, sliced)
    if best is None:
        raise ValueError("no candidate plan within max_peak")
    return best[1], best[2], best[0][0], best[0][1]


def fitted_plan(legs, trials, seed, open_edges, n_outputs, n_bits, max_peak,
                settings=((1.0, 0.6), (0.75, 0.3), (0.75, 0.6), (0.5, 0.6), (0.25, 0.3), (1.0, 1.0), (1.0, 0.2)),
                max_pair_peak=None, max_slices=24):
    """Seeded greedy candidates (as level_aware_plan), each sliced by tree trimming with as few bonds as
    keep every intermediate within max_peak legs, and those stored per (slice, bitstring) pair within
    max_pair_peak when given (Sec. III-A: slicing trades memory for more contractions); the candidate
    with the smallest executed_time for n_bits bitstrings wins (ties: fewer sliced bonds, earlier
    candidate).  Returns (order, sliced, estimated seconds)."""
    rng = SplitMix64(seed)
    orders = [_greedy(legs)]
    for alpha, temp in settings:
        for _ in range(trials):
            orders.append(_greedy(legs, rng, temp, alpha))
    best = None
    for k, order in enumerate(orders):
        sliced = []
        while len(sliced) < max_slices and (plan_cost(legs, order, sliced)[0] > max_peak or (
                max_pair_peak is not None and pair_peak(legs, order, sliced, n_outputs) > max_pair_peak)):
            sliced = tree_trim_slices(legs, order, len(sliced) + 1, seed + k, open_edges)
        if plan_cost(legs, order, sliced)[0] > max_peak:
            continue
        t = executed_time(legs, order, sliced, n_outputs, n_bits)
        key = (t, len(sliced), k)
        if best is None or key < best[0]:
            best = (key, order, sliced)
    return best[1], best[2], best[0][0]


def pair_peak(legs, order, sliced, n_outputs):
    """Largest rank (legs, fixed bonds removed) of an intermediate that an output bit reaches: those are
    stored once per (slice, bitstring) pair, so they set the memory a batch of pairs needs."""
    sl = frozenset(sliced)
    first_out = len(legs) - n_outputs
    out_wires = frozenset(e for t in range(first_out, len(legs)) for e in legs[t])
    fixed = sl | out_wires
    sets = [frozenset(l) for l in legs]
    by_bits = [bool(out_wires & sets[t]) for t in range(len(legs))]
    peak = 0
    for a, b in order:
        s = sets[a] ^ sets[b]
        d = by_bits[a] or by_bits[b]
        sets.append(s)
        by_bits.append(d)
        if d:
            peak = max(peak, len(s - fixed))
    return peak


def _order_to_tree(n_leaves, order):
    return {n_leaves + t: (a, b) for t, (a, b) in enumerate(order)}, n_leaves + len(order) - 1


def _tree_to_order(n_leaves, children, root):
    """SSA order of a contraction tree: children before parents, left subtree first."""
    order, new_id = [], {}
    stack = [(root, False)]
    while stack:
        node, done = stack.pop()
        if node < n_leaves:
            continue
        a, b = children[node]
        if done:
            order.append((new_id.get(a, a), new_id.get(b, b)))
            new_id[node] = n_leaves + len(order) - 1
        else:
            stack.append((node, True))
            stack.append((b, False))
            stack.append((a, False))
    return order


def local_search_plan(legs, order, sliced, n_outputs, n_bits, max_peak, iters, seed, objective="flops",
                      max_pair_peak=None):
    """Local optimisation of a plan (this project's own step beyond the paper's planner): seeded
    random rotations of the contraction tree, ((A, B), C) -> ((A, C), B), each kept when the plan
    costs less per call with every intermediate within max_peak legs; the sliced bonds stay as given.
    objective "flops": executed flops per call (executed_cost); "time": the roofline estimate of
    executed_time; or a function (legs, order, sliced, n_outputs, n_bits) -> cost.  max_pair_peak, when
    given, also bounds the intermediates stored per (slice, bitstring) pair (pair_peak).  Returns (order,
    cost, accepted moves).
    """
    n = len(legs)
    children, root = _order_to_tree(n, order)
    internal = sorted(children)
    if callable(objective):
        cost_of = objective
    elif objective == "flops":
        cost_of = executed_cost
    elif objective == "time":
        cost_of = executed_time
    else:
        raise ValueError(f"unknown objective {objective!r}")
    best = cost_of(legs, order, sliced, n_outputs, n_bits)
    rng = SplitMix64(seed)
    accepted = 0
    for _ in range(iters):
        p = internal[rng.randint(len(internal))]
        a, b = children[p]
        x, y = (a, b) if rng.randint(2) == 0 else (b, a)  # x: the child to open, y: its sibling
        if x < n:
            continue
        xa, xb = children[x]
        keep, move = (xa, xb) if rng.randint(2) == 0 else (xb, xa)
        old_p, old_x = children[p], children[x]
        children[x], children[p] = (keep, y), (x, move)
        cand = _tree_to_order(n, children, root)
        ok = plan_cost(legs, cand, sliced)[0] <= max_peak and (
            max_pair_peak is None or pair_peak(legs, cand, sliced, n_outputs) <= max_pair_peak)
        cost = cost_of(legs, cand, sliced, n_outputs, n_bits) if ok else None
        if cost is not None and cost < best:
            best, accepted = cost, accepted + 1
        else:
            children[p], children[x] = old_p, old_x
    return _tree_to_order(n, children, root), best, accepted


def sliceable_bonds(legs, n_outputs, open_edges=()):
    """Bonds a plan may slice: bonds between two tensors, other than the final wires of closed qubits
    (their output vectors fix them already) and open legs."""
    deg = {}
    for L in legs:
        for e in L:
            deg[e] = deg.get(e, 0) + 1
    no_slice = set(open_edges) | {legs[t][0] for t in range(len(legs) - n_outputs, len(legs))}
    return sorted(e for e, d in deg.items() if d == 2 and e not in no_slice)


def anneal_plan(legs, order, sliced, n_outputs, n_bits, max_peak, iters, seed, objective, candidates=(),
                p_swap=0.0, t_start=3e-3, t_end=1e-5):
    """Simulated annealing over the contraction tree and the choice of sliced bonds (this project's own
    planner step; the paper's planner fixes the sliced bonds by tree trimming, which minimises the
    largest intermediate, not the work a call executes once slice-invariant steps run once).

    Each iteration draws a uniform u for the acceptance test, then with probability p_swap replaces one
    sliced bond (a seeded draw) by a bond of `candidates` not sliced yet -- the number of sliced bonds,
    and so of slices, stays -- and otherwise applies one seeded tree rotation ((A, B), C) -> ((A, C), B)
    as local_search_plan does.  A candidate whose intermediates all fit max_peak legs is accepted when
    it costs no more, or else when u < exp(-(cost - current) / T), with T falling geometrically from
    t_start to t_end times the starting cost over the iterations.  objective: a function (legs, order,
    sliced, n_outputs, n_bits) -> cost.  Returns (order, sliced, cost, accepted moves) of the cheapest
    plan visited."""
    n = len(legs)
    children, root = _order_to_tree(n, order)
    internal = sorted(children)
    cands = list(candidates)
    sliced = list(sliced)
    cur = objective(legs, order, sliced, n_outputs, n_bits)
    c0 = cur
    best, best_order, best_sliced = cur, list(order), list(sliced)
    rng = SplitMix64(seed)
    accepted = 0
    for i in range(iters):
        T = c0 * t_start * (t_end / t_start) ** (i / max(1, iters - 1))
        u = rng.uniform()
        if rng.uniform() < p_swap:
            j = rng.randint(len(sliced))
            e = cands[rng.randint(len(cands))]
            if e in sliced:
                continue
            new_sl = list(sliced)
            new_sl[j] = e
            cand = _tree_to_order(n, children, root)
            c = objective(legs, cand, new_sl, n_outputs, n_bits) if plan_cost(legs, cand, new_sl)[0] <= max_peak \
                else None
            if c is not None and (c <= cur or u < math.exp(-(c - cur) / T)):
                cur, sliced = c, new_sl
                accepted += 1
                if c < best:
                    best, best_order, best_sliced = c, cand, list(sliced)
            continue
        p = internal[rng.randint(len(internal))]
        a, b = children[p]
        x, y = (a, b) if rng.randint(2) == 0 else (b, a)  # x: the child to open, y: its sibling
        if x < n:
            continue
        xa, xb = children[x]
        keep, move = (xa, xb) if rng.randint(2) == 0 else (xb, xa)
        old_p, old_x = children[p], children[x]
        children[x], children[p] = (keep, y), (x, move)
        cand = _tree_to_order(n, children, root)
        c = objective(legs, cand, sliced, n_outputs, n_bits) if plan_cost(legs, cand, sliced)[0] <= max_peak else None
        if c is not None and (c <= cur or u < math.exp(-(c - cur) / T)):
            cur = c
            accepted += 1
            if c < best:
                best, best_order, best_sliced = c, cand, list(sliced)
        else:
            children[p], children[x] = old_p, old_x
    return best_order, best_sliced, best, accepted


def sweep_order(legs, n_qubits, n_outputs, gate_qubits):
    """A state-vector-like contraction order (this project's own starting point for annealing): the
    gates that touch no closed output wire are contracted onto the tensors holding their qubits in
    circuit order, one-qubit gates first merged with the next two-qubit gate on their qubit, so the
    growing tensor never has more legs than there are qubits; the gates of the final layer with their
    output vectors come last.  Every step below the final layer reaches no output bit, so without
    sliced bonds it runs once per call and each bitstring adds only the final layer's contractions.
    gate_qubits: the qubits of each gate, in the order network_legs was given them."""
    n = len(legs)
    first_out = n - n_outputs
    out_of = {legs[t][0]: t for t in range(first_out, n)}
    order = []

    def join(a, b):
        order.append((a, b))
        return n + len(order) - 1

    holder = list(range(n_qubits))  # tensor holding each qubit's wire (its input tensor at first)
    pend = {}                       # one-qubit gates on a qubit not yet merged into a larger gate
    gates = range(n_qubits, first_out)
    final = [t for t in gates if any(e in out_of for e in legs[t])]
    fset = set(final)

    def apply(cur, qs):
        for q in qs:
            if q in pend:
                cur = join(cur, pend.pop(q))
        hs = []
        for q in qs:
            if holder[q] not in hs:
                hs.append(holder[q])
        for h in hs:
            cur = join(h, cur)
        for q in range(n_qubits):
            if holder[q] in hs:
                holder[q] = cur

    for t in gates:
        if t in fset:
            continue
        qs = gate_qubits[t - n_qubits]
        if len(qs) == 1:
            pend[qs[0]] = join(pend[qs[0]], t) if qs[0] in pend else t
        else:
            apply(t, qs)
    for f in final:
        qs = gate_qubits[f - n_qubits]
        cur = f
        for e in legs[f][:len(qs)]:
            if e in out_of:
                cur = join(cur, out_of.pop(e))
        apply(cur, qs)
    for q in sorted(pend):  # open qubits' trailing one-qubit gates
        apply(pend.pop(q), [q])
    for q in range(n_qubits):  # closed qubits without gates: the output vector meets the input
        if q in out_of:
            apply(out_of.pop(q), [q])
    roots = sorted(set(holder))
    while len(roots) > 1:
        roots = [join(roots[0], roots[1])] + roots[2:]
    if len(order) != n - 1:
        raise ValueError("sweep_order: the network is not one contraction tree")
    return order
