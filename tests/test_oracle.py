"""Pins for the complex128 oracle against facts the paper and mathematics fix.

Every check here compares the oracle with something other than itself:
closed forms (GHZ, product states), unitarity, the other oracle (state vector
vs plan einsum: two independent algorithms), the slicing identity of Eq. 2,
the order-count formula of Sec. III-A with brute force over every pairwise
order, and mirror circuits U U^dagger.  A few tests plant a plausible mistake
in the oracle and check that a pin catches it.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import einsum as oe
from qxgen import circuits as C
from qxgen.plan import greedy_order, network_legs, tree_trim_slices
from qxgen.workloads import make_plan


def _plan(circ, open_mask=None, n_slice=0, seed=1):
    n = circ.n_qubits
    om = np.zeros(n, np.uint8) if open_mask is None else np.asarray(open_mask, np.uint8)
    order, sliced, _, _ = make_plan(circ, om, n_slice, seed)
    return om, order, sliced


def _all_bits(n):
    return np.array([[(i >> (n - 1 - q)) & 1 for q in range(n)] for i in range(1 << n)], dtype=np.uint8)


# --- inputs: gate matrices --------------------------------------------------------------------

def test_gate_matrices_unitary_and_fsim_swap_phase():
    for u in list(C.ONE_QUBIT_SET) + [C.FSIM_SYC, C.HADAMARD, C.CNOT]:
        assert np.allclose(u.conj().T @ u, np.eye(u.shape[0]), atol=1e-15)
    # fSim(pi/2, .) sends |01> to -i|10> (iSWAP-like exchange)
    out = C.FSIM_SYC @ np.array([0, 1, 0, 0], dtype=np.complex128)
    assert np.allclose(out, [0, 0, -1j, 0], atol=1e-15)
    assert np.isclose(C.FSIM_SYC[3, 3], np.exp(-1j * np.pi / 6))


def test_splitmix64_reference_outputs():
    # published splitmix64 (Vigna's reference C implementation) seeded with 0
    r = C.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4


def test_grid_circuit_counts():
    circ = C.random_grid_circuit(3, 4, 8, 1001)
    assert sum(len(g.qubits) == 1 for g in circ.gates) == 96
    assert sum(len(g.qubits) == 2 for g in circ.gates) == 34
    # no qubit gets the same single-qubit gate in consecutive cycles
    per_q = {}
    for g in circ.gates:
        if len(g.qubits) == 1:
            per_q.setdefault(g.qubits[0], []).append(g.name)
    for names in per_q.values():
        assert all(a != b for a, b in zip(names, names[1:]))


# --- GHZ closed form (circuit named in Table II) -----------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_ghz_statevector(n):
    psi = oracle.statevector(n, C.gates_to_records(C.ghz_circuit(n)))
    want = np.zeros(1 << n, np.complex128)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.allclose(psi, want, atol=1e-14)


@pytest.mark.parametrize("n,n_slice", [(3, 0), (5, 2), (8, 3)])
def test_ghz_einsum(n, n_slice):
    circ = C.ghz_circuit(n)
    om, order, sliced = _plan(circ, n_slice=n_slice)
    bits = np.array([[0] * n, [1] * n, [1] + [0] * (n - 1), [0] * (n - 1) + [1]], np.uint8)
    amps = oe.amplitudes(n, C.gates_to_records(circ), om, order, sliced, bits)[:, 0]
    s = 1 / math.sqrt(2)
    assert np.allclose(amps, [s, s, 0, 0], atol=1e-14)


def test_ghz_open_legs_give_the_state():
    n = 4
    circ = C.ghz_circuit(n)
    om = np.ones(n, np.uint8)
    _, order, sliced = _plan(circ, om, n_slice=1)
    vec = oe.amplitudes(n, C.gates_to_records(circ), om, order, sliced, np.zeros((1, n), np.uint8))[0]
    want = np.zeros(1 << n)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.allclose(vec, want, atol=1e-14)


# --- product-state closed form ------------------------------------------------------------------

def test_product_state_closed_form_both_oracles():
    n = 6
    circ = C.product_circuit(n, 3, seed=77)
    recs = C.gates_to_records(circ)
    v = [np.eye(2, dtype=np.complex128) for _ in range(n)]
    for g in circ.gates:
        v[g.qubits[0]] = g.matrix @ v[g.qubits[0]]
    bits = C.random_bitstrings(n, 12, 5)
    want = np.array([np.prod([v[q][x[q], 0] for q in range(n)]) for x in bits])
    sv = oracle.sv_amplitudes(n, recs, None, bits)[:, 0]
    om, order, sliced = _plan(circ, n_slice=0)
    es = oe.amplitudes(n, recs, om, order, sliced, bits)[:, 0]
    assert np.allclose(sv, want, atol=1e-14)
    assert np.allclose(es, want, atol=1e-14)


# --- unitarity ----------------------------------------------------------------------------------

def test_unitarity_statevector():
    circ = C.random_grid_circuit(3, 4, 8, 1001)
    psi = oracle.statevector(12, C.gates_to_records(circ))
    assert abs(np.vdot(psi, psi).real - 1) < 1e-12


def test_unitarity_einsum_all_bitstrings():
    circ = C.random_grid_circuit(2, 3, 6, 11)
    om, order, sliced = _plan(circ, n_slice=2)
    amps = oe.amplitudes(6, C.gates_to_records(circ), om, order, sliced, _all_bits(6))[:, 0]
    assert abs(np.sum(np.abs(amps) ** 2) - 1) < 1e-12


# --- two independent algorithms agree -----------------------------------------------------------

@pytest.mark.parametrize("rows,cols,depth,n_open,n_slice", [(3, 3, 6, 0, 0), (3, 3, 8, 2, 3), (2, 4, 10, 3, 2)])
def test_statevector_equals_einsum(rows, cols, depth, n_open, n_slice):
    n = rows * cols
    circ = C.random_grid_circuit(rows, cols, depth, 100 + depth)
    om = np.zeros(n, np.uint8)
    om[n - n_open:] = 1
    _, order, sliced = _plan(circ, om, n_slice)
    recs = C.gates_to_records(circ)
    bits = C.random_bitstrings(n, 6, 9)
    a = oracle.sv_amplitudes(n, recs, om, bits)
    b = oe.amplitudes(n, recs, om, order, sliced, bits)
    assert np.max(np.abs(a - b)) < 1e-13


def test_sliced_equals_unsliced_eq2():
    circ = C.random_grid_circuit(3, 4, 8, 1001)
    recs = C.gates_to_records(circ)
    om = np.zeros(12, np.uint8)
    legs, _, open_edges = network_legs(12, [g.qubits for g in circ.gates], om)
    order = greedy_order(legs)
    sliced = tree_trim_slices(legs, order, 4, 3)
    bits = C.random_bitstrings(12, 4, 3)
    full = oe.amplitudes(12, recs, om, order, [], bits)
    parts = oe.amplitudes(12, recs, om, order, sliced, bits)
    assert np.max(np.abs(full - parts)) < 1e-14
    # the slices really differ (each is a different smaller network)
    r0 = oe.contract_once(12, recs, om, order, sliced, 0, bits[0])
    r1 = oe.contract_once(12, recs, om, order, sliced, 5, bits[0])
    assert abs(r0[0] - r1[0]) > 1e-6


# --- order count N!(N-1)!/2^(N-1) and order independence by brute force ----------------------

def _all_orders(ids, next_id):
    if len(ids) == 1:
        yield []
        return
    for a, b in itertools.combinations(sorted(ids), 2):
        rest = [i for i in ids if i not in (a, b)] + [next_id]
        for tail in _all_orders(rest, next_id + 1):
            yield [(a, b)] + tail


@pytest.mark.parametrize("extra_1q", [0, 1])
def test_every_pairwise_order_gives_the_same_amplitude(extra_1q):
    circ = C.Circuit(2)
    circ.append((0, 1), C.FSIM_SYC)
    circ.append((0,), C.SQRT_W)
    if extra_1q:
        circ.append((1,), C.SQRT_Y)
    recs = C.gates_to_records(circ)
    n_t = 2 + len(circ.gates) + 2
    orders = list(_all_orders(list(range(n_t)), n_t))
    assert len(orders) == math.factorial(n_t) * math.factorial(n_t - 1) // 2 ** (n_t - 1)
    bit = np.array([[1, 0]], np.uint8)
    want = oracle.sv_amplitudes(2, recs, None, bit)[0, 0]
    assert abs(want) > 0.1
    for order in orders:
        got = oe.amplitudes(2, recs, None, order, [], bit)[0, 0]
        assert abs(got - want) < 1e-14


# --- mirror circuits ------------------------------------------------------------------------------

@pytest.mark.parametrize("rows,cols,depth,n_slice", [(4, 4, 4, 2), (6, 6, 2, 2)])
def test_mirror_circuit_returns_to_zero(rows, cols, depth, n_slice):
    n = rows * cols
    u = C.random_grid_circuit(rows, cols, depth, 55)
    circ = u.then(u.inverse())
    om, order, sliced = _plan(circ, n_slice=n_slice)
    bits = np.concatenate([np.zeros((1, n), np.uint8), C.random_bitstrings(n, 2, 8)])
    amps = oe.amplitudes(n, C.gates_to_records(circ), om, order, sliced, bits)[:, 0]
    assert abs(amps[0] - 1) < 1e-12
    assert np.all(np.abs(amps[1:]) < 1e-12)


# --- compensated slice sum -----------------------------------------------------------------------

def test_neumaier_matches_fsum():
    rng = np.random.default_rng(3)
    xs = rng.standard_normal(2000) * 10.0 ** rng.integers(-12, 12, 2000)
    acc = oe._Neumaier(1)
    for x in xs:
        acc.add(np.array([x]))
    assert acc.value()[0] == math.fsum(xs)


# --- planted mistakes: the pins above catch each one --------------------------------------------

def test_planted_transposed_gate_is_caught(monkeypatch):
    orig = oe._gate_matrix
    monkeypatch.setattr(oe, "_gate_matrix", lambda rec: (orig(rec)[0], orig(rec)[1].T))
    n = 6
    circ = C.product_circuit(n, 3, seed=77)
    om, order, sliced = _plan(circ)
    bits = C.random_bitstrings(n, 4, 5)
    recs = C.gates_to_records(circ)
    assert np.max(np.abs(oe.amplitudes(n, recs, om, order, sliced, bits) -
                         oracle.sv_amplitudes(n, recs, None, bits))) > 1e-3


def test_planted_wrong_slice_bit_is_caught(monkeypatch):
    orig = oe._fix
    monkeypatch.setattr(oe, "_fix", lambda arr, legs, e, v: orig(arr, legs, e, 0))
    circ = C.random_grid_circuit(3, 3, 6, 106)
    om, order, sliced = _plan(circ, n_slice=3)
    bits = C.random_bitstrings(9, 3, 9)
    recs = C.gates_to_records(circ)
    assert np.max(np.abs(oe.amplitudes(9, recs, om, order, sliced, bits) -
                         oracle.sv_amplitudes(9, recs, None, bits))) > 1e-3


def test_planted_dropped_compensation_is_caught(monkeypatch):
    class Plain(oe._Neumaier):
        def add(self, x):
            self.s = self.s + x
    monkeypatch.setattr(oe, "_Neumaier", Plain)
    xs = [1e16, 1.0, -1e16, 1.0]
    acc = oe._Neumaier(1)
    for x in xs:
        acc.add(np.array([x]))
    assert acc.value()[0] != math.fsum(xs)


def test_porter_thomas_second_moment_of_deep_random_circuits():
    """Deep random circuits scramble: p = 2^n |amp|^2 over all x has mean 1 (unitarity) and second
    moment near 2 (the exponential law of Porter and Thomas); shallow ones are far from it."""
    n = 16
    zero = np.zeros((1, n), np.uint8)
    moments = {}
    for depth in (2, 16):
        circ = C.random_grid_circuit(4, 4, depth, 4242)
        a = oracle.sv_amplitudes(n, C.gates_to_records(circ), np.ones(n, np.uint8), zero).reshape(-1)
        p = (1 << n) * np.abs(a) ** 2
        assert abs(p.mean() - 1.0) < 1e-10
        moments[depth] = float((p ** 2).mean())
    assert abs(moments[16] - 2.0) < 0.1
    assert moments[2] > 3.0


def test_cancelling_slices_need_the_compensated_sum():
    """The case that pins the device's compensated slice sum: per-slice values X, 1, -X, -1 in slice
    order (checked through the oracle one slice at a time); a plain FP64 running sum gives -1, the
    oracle's compensated sum and math.fsum give the exact 0."""
    from ._util import cancelling_slices_case
    circ, om, order, sliced, bits = cancelling_slices_case()
    recs = C.gates_to_records(circ)
    per = [oe.amplitudes(2, recs, om, order, sliced, bits, slices=[s])[0, 0] for s in range(4)]
    X = 2.0 ** 60
    assert [p.real for p in per] == [X, 1.0, -X, -1.0] and all(p.imag == 0 for p in per)
    naive = 0.0
    for p in per:
        naive += p.real
    assert naive == -1.0
    assert math.fsum(p.real for p in per) == 0.0
    assert oe.amplitudes(2, recs, om, order, sliced, bits)[0, 0] == 0.0
    assert oracle.sv_amplitudes(2, recs, om, bits)[0, 0] == 0.0


def test_parity_bounds_catch_a_concentrated_error():
    """The tests' two parity bounds: independent errors at 80% of the l2 tolerance pass both; the
    same l2 error put into one amplitude passes the l2 bound but fails the element-wise one."""
    from ._util import TOL_C64, assert_parity, tol_elem
    rng = np.random.default_rng(5)
    for n in (64, 256, 4096):
        ref = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / np.sqrt(2 * n)
        noise = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        noise *= 0.8 * TOL_C64 * np.linalg.norm(ref) / np.linalg.norm(noise)
        assert_parity(ref + noise, ref)
        one = np.zeros(n, complex)
        one[n // 3] = 0.8 * TOL_C64 * np.linalg.norm(ref)
        with pytest.raises(AssertionError):
            assert_parity(ref + one, ref)
        assert tol_elem(n) < 0.8 * TOL_C64 * np.sqrt(n)
