"""Oracle: plan-following pairwise contraction in complex128 (numpy).

TEST INFRASTRUCTURE ONLY.  Part of the independent CPU oracle; only the
tests, the smoke check and the CPU-baseline leg of the benchmark use it.

What it computes, step by step in the paper's terms:

1. Circuit -> tensor network (Sec. II): every qubit starts as the rank-1
   tensor |0> = (1, 0); a single-qubit gate is its 2x2 matrix as a rank-2
   tensor; a two-qubit gate's 4x4 matrix is reshaped to a rank-4 2x2x2x2
   tensor; each gate is attached to the open legs of its qubits in circuit
   order.
2. Closing the outputs (Sec. II): every qubit that is not left open gets the
   rank-1 tensor <x_q| = e_{x_q}; contracting the network then yields
   <x|C|0> (with the open qubits' legs left as the result's axes).
3. Pairwise contraction (Sec. III-A): the network is contracted as the given
   sequence of pairwise products; each product sums over the bonds the two
   tensors share (numpy.tensordot, a library matrix product, does each one).
4. Slicing (Sec. III-A, Eq. 2): each sliced bond is fixed to one of its
   values, the smaller network is contracted, and the results for all
   values are summed.  Slice s gives bond sliced[j] the value of bit j of s.
   The sum runs in complex128 with Neumaier compensation per component.

Canonical labels (shared by the C-ABI so both sides read the same plan):
tensor ids 0..n-1 are the inputs, n..n+G-1 the gates in list order, then one
output tensor per closed qubit in increasing qubit order; bond ids 0..n-1 are
the input wires, then each gate's output legs in creation order (q0 first).
A plan step (i, j) creates the tensor with the next free id.

Reading taken where the paper's Eq. 2 is garbled: the inner sum runs over
every bond except the sliced one, for a fixed value of the sliced bond.

Parity pins: tests/test_oracle.py (GHZ, product states, unitarity, the
state-vector oracle, sliced == unsliced, order independence by brute force,
mirror circuits).
"""
from __future__ import annotations

import numpy as np


def _gate_matrix(rec):
    nq = int(rec["nq"])
    d = 2 if nq == 1 else 4
    m = np.asarray(rec["re"][: d * d], dtype=np.float64) + 1j * np.asarray(rec["im"][: d * d], dtype=np.float64)
    return nq, m.reshape(d, d)


def build_network(n_qubits, gates, open_mask=None):
    """Tensors of the circuit network before outputs are attached.

    Returns (tensors, closed_wires, open_wires) where tensors is a list of
    [array, legs] for inputs and gates (canonical ids 0..n+G-1),
    closed_wires[q] is the last bond on closed qubit q (None when open) and
    open_wires lists the last bonds of the open qubits in qubit order.
    """
    if open_mask is None:
        open_mask = np.zeros(n_qubits, dtype=np.uint8)
    wire = list(range(n_qubits))
    tensors = [[np.array([1.0, 0.0], dtype=np.complex128), [q]] for q in range(n_qubits)]
    next_edge = n_qubits
    for rec in gates:
        nq, u = _gate_matrix(rec)
        qs = [int(rec["q"][0])] + ([int(rec["q"][1])] if nq == 2 else [])
        for q in qs:
            if not 0 <= q < n_qubits:
                raise ValueError("gate qubit out of range")
        if nq == 2 and qs[0] == qs[1]:
            raise ValueError("two-qubit gate on one qubit")
        outs = list(range(next_edge, next_edge + nq))
        next_edge += nq
        arr = u.reshape((2,) * (2 * nq))     # T[o0, (o1,) i0, (i1)] = U[row(o), col(i)]
        tensors.append([arr, outs + [wire[q] for q in qs]])
        for q, e in zip(qs, outs):
            wire[q] = e
    closed = [None if open_mask[q] else wire[q] for q in range(n_qubits)]
    opened = [wire[q] for q in range(n_qubits) if open_mask[q]]
    return tensors, closed, opened


def _fix(arr, legs, edge, value):
    ax = legs.index(edge)
    return np.take(arr, value, axis=ax), legs[:ax] + legs[ax + 1:]


def contract_once(n_qubits, gates, open_mask, order, sliced, slice_index, bitstring):
    """One sliced network for one bitstring: returns the open-leg vector."""
    tensors, closed, opened = build_network(n_qubits, gates, open_mask)
    for q in range(n_qubits):
        if closed[q] is not None:
            v = np.zeros(2, dtype=np.complex128)
            v[int(bitstring[q])] = 1.0
            tensors.append([v, [closed[q]]])
    n_t = len(tensors)
    if len(order) != n_t - 1:
        raise ValueError("plan must contract the whole network")
    for j, e in enumerate(sliced):
        val = (slice_index >> j) & 1
        holders = [t for t in tensors if e in t[1]]
        if len(holders) != 2:
            raise ValueError("sliced bond must join two tensors")
        for t in holders:
            t[0], t[1] = _fix(t[0], t[1], e, val)
    pool = {i: t for i, t in enumerate(tensors)}
    nid = n_t
    for (a, b) in order:
        a, b = int(a), int(b)
        if a not in pool or b not in pool or a == b:
            raise ValueError("plan step uses a missing or consumed tensor")
        A, la = pool.pop(a)
        B, lb = pool.pop(b)
        shared = [e for e in la if e in lb]
        C = np.tensordot(A, B, axes=([la.index(e) for e in shared], [lb.index(e) for e in shared]))
        lc = [e for e in la if e not in shared] + [e for e in lb if e not in shared]
        pool[nid] = [C, lc]
        nid += 1
    (root, legs), = pool.values()
    if sorted(legs) != sorted(opened):
        raise ValueError("result legs do not match the open qubits")
    root = np.transpose(root, [legs.index(e) for e in opened]) if opened else root
    return np.asarray(root, dtype=np.complex128).reshape(-1)


class _Neumaier:
    """Compensated running sum of complex128 arrays (Neumaier 1974), per component."""

    def __init__(self, shape):
        self.s = np.zeros(shape, dtype=np.float64)
        self.c = np.zeros(shape, dtype=np.float64)

    def add(self, x):
        t = self.s + x
        big = np.abs(self.s) >= np.abs(x)
        self.c += np.where(big, (self.s - t) + x, (x - t) + self.s)
        self.s = t

    def value(self):
        return self.s + self.c


def amplitudes(n_qubits, gates, open_mask, order, sliced, bitstrings, slices=None):
    """Amplitudes summed over `slices` (default: all 2^len(sliced) of them).

    Returns a complex128 array of shape (n_bits, 2^n_open); the first open qubit
    is the most significant bit of the open index.
    """
    if open_mask is None:
        open_mask = np.zeros(n_qubits, dtype=np.uint8)
    bitstrings = np.asarray(bitstrings, dtype=np.uint8).reshape(-1, n_qubits)
    if np.any(bitstrings > 1):
        raise ValueError("bitstrings must be 0/1")
    n_open = int(np.sum(np.asarray(open_mask) != 0))
    if slices is None:
        slices = range(1 << len(sliced))
    out = np.zeros((len(bitstrings), 1 << n_open), dtype=np.complex128)
    for bi, x in enumerate(bitstrings):
        re, im = _Neumaier(1 << n_open), _Neumaier(1 << n_open)
        for s in slices:
            r = contract_once(n_qubits, gates, open_mask, order, sliced, s, x)
            re.add(r.real)
            im.add(r.imag)
        out[bi] = re.value() + 1j * im.value()
    return out
