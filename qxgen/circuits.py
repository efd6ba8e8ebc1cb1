"""Seeded synthetic circuits and bitstrings (input generation only).

This module produces the inputs that both the CUDA path and the oracle
consume: gate lists for random grid circuits of the Sycamore style and
uniformly random output bitstrings.  It holds no contraction arithmetic.

The paper's workloads are the random quantum circuits of Boixo et al. on a
two-dimensional qubit grid with layers of gates on all qubits (Sec. IV-B).
The circuits here follow the same recipe with the Sycamore gate set:

* every cycle applies one single-qubit gate per qubit drawn from
  {sqrt(X), sqrt(Y), sqrt(W)}, never the same gate a qubit got in the
  previous cycle (the first cycle draws uniformly from all three);
* then fSim(theta=pi/2, phi=pi/6) on every coupler of one of four
  nearest-neighbour patterns, cycled A, B, C, D:
  A = horizontal (r,c)-(r,c+1) with c even, B = horizontal with c odd,
  C = vertical (r,c)-(r+1,c) with r even, D = vertical with r odd.
* a depth-d circuit is d such cycles, with no trailing single-qubit layer.

Qubit q sits at row q // cols, column q % cols.  Gates carry their explicit
matrices, row-major, in the basis |q0 q1> where q0 is the first target.

Randomness comes from splitmix64 (Steele, Lea and Flood, 2014): the state
advances by 0x9E3779B97F4A7C15 and each output is the state passed through
the published two-multiply finaliser.  Integer draws in [0, k) take the
output modulo k; the bias (< k / 2^64) is irrelevant here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator (Steele, Lea, Flood: 'Fast splittable PRNGs')."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def randint(self, k: int) -> int:
        """Uniform integer in [0, k)."""
        return self.next_u64() % k

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


# --- gate matrices (public Sycamore conventions) -------------------------------------------

_S = 1.0 / math.sqrt(2.0)
SQRT_X = np.array([[1, -1j], [-1j, 1]], dtype=np.complex128) * _S
SQRT_Y = np.array([[1, -1], [1, 1]], dtype=np.complex128) * _S
SQRT_W = np.array([[1, -np.exp(1j * np.pi / 4)], [np.exp(-1j * np.pi / 4), 1]],
                  dtype=np.complex128) * _S
ONE_QUBIT_SET = (SQRT_X, SQRT_Y, SQRT_W)
ONE_QUBIT_NAMES = ("sqrtX", "sqrtY", "sqrtW")
HADAMARD = np.array([[1, 1], [1, -1]], dtype=np.complex128) * _S
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) in the basis |00>, |01>, |10>, |11>."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)


FSIM_SYC = fsim(math.pi / 2, math.pi / 6)


@dataclass
class Gate:
    qubits: tuple            # (q0,) or (q0, q1)
    matrix: np.ndarray       # 2x2 or 4x4 complex128, row-major, basis |q0 q1>
    name: str = ""


@dataclass
class Circuit:
    n_qubits: int
    gates: list = field(default_factory=list)
    rows: int = 0
    cols: int = 0
    depth: int = 0
    seed: int = 0

    def append(self, qubits, matrix, name=""):
        self.gates.append(Gate(tuple(int(q) for q in qubits), np.asarray(matrix, np.complex128), name))
        return self

    def inverse(self) -> "Circuit":
        """U^dagger: the gates in reverse order, each conjugate-transposed."""
        inv = Circuit(self.n_qubits, rows=self.rows, cols=self.cols, depth=self.depth, seed=self.seed)
        for g in reversed(self.gates):
            inv.append(g.qubits, g.matrix.conj().T, g.name + "^dag")
        return inv

    def then(self, other: "Circuit") -> "Circuit":
        out = Circuit(self.n_qubits, list(self.gates) + list(other.gates), self.rows, self.cols,
                      self.depth + other.depth, self.seed)
        return out


# C layout of one gate record, shared by the C-ABI header and the oracle:
# struct { int32 nq; int32 q[2]; double re[16]; double im[16]; }  (272 bytes)
GATE_DTYPE = np.dtype([("nq", "<i4"), ("q", "<i4", (2,)), ("pad", "<i4"),
                       ("re", "<f8", (16,)), ("im", "<f8", (16,))])
assert GATE_DTYPE.itemsize == 272


def gates_to_records(circ: Circuit) -> np.ndarray:
    """Pack a circuit into the 272-byte gate records both sides read."""
    rec = np.zeros(len(circ.gates), dtype=GATE_DTYPE)
    for i, g in enumerate(circ.gates):
        nq = len(g.qubits)
        rec[i]["nq"] = nq
        rec[i]["q"][0] = g.qubits[0]
        rec[i]["q"][1] = g.qubits[1] if nq == 2 else -1
        m = g.matrix.reshape(-1)
        rec[i]["re"][: m.size] = m.real
        rec[i]["im"][: m.size] = m.imag
    return rec


# --- grid geometry -------------------------------------------------------------------------

def near_square_shape(n: int) -> tuple:
    """rows = floor(sqrt(n)), cols = ceil(n / rows); a leftover fills a partial last row."""
    rows = max(1, math.isqrt(n))
    cols = -(-n // rows)
    return rows, cols


def coupler_pattern(rows: int, cols: int, n: int, pattern: int) -> list:
    """Couplers of pattern 0..3 (A, B, C, D) as (q0, q1) with q0 < q1, sorted by q0."""
    pairs = []
    for q in range(n):
        r, c = divmod(q, cols)
        if pattern in (0, 1):
            if c % 2 == pattern and c + 1 < cols and q + 1 < n:
                pairs.append((q, q + 1))
        else:
            if r % 2 == pattern - 2 and q + cols < n:
                pairs.append((q, q + cols))
    return pairs


def random_grid_circuit(rows: int, cols: int, depth: int, seed: int, n: int | None = None) -> Circuit:
    """Seeded Sycamore-style random circuit on a rows x cols grid (n <= rows*cols qubits)."""
    if n is None:
        n = rows * cols
    rng = SplitMix64(seed)
    circ = Circuit(n, rows=rows, cols=cols, depth=depth, seed=seed)
    prev = [-1] * n
    for t in range(depth):
        for q in range(n):
            if prev[q] < 0:
                k = rng.randint(3)
            else:
                others = [i for i in range(3) if i != prev[q]]
                k = others[rng.randint(2)]
            prev[q] = k
            circ.append((q,), ONE_QUBIT_SET[k], ONE_QUBIT_NAMES[k])
        for (a, b) in coupler_pattern(rows, cols, n, t % 4):
            circ.append((a, b), FSIM_SYC, "fsim")
    return circ


def random_bitstrings(n_qubits: int, count: int, seed: int) -> np.ndarray:
    """count x n_qubits uint8 array of uniform 0/1 values."""
    rng = SplitMix64(seed)
    out = np.zeros((count, n_qubits), dtype=np.uint8)
    for i in range(count):
        for q in range(n_qubits):
            out[i, q] = rng.next_u64() >> 63
    return out


def splitmix64_stream(seed: int, count: int) -> np.ndarray:
    """The first `count` splitmix64 outputs of `seed`, vectorised.

    Output k (k = 1, 2, ...) is the finaliser applied to seed + k * gamma, so
    the stream is the one SplitMix64(seed).next_u64() produces.
    """
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def sampler_draws(n_qubits: int, count: int, seed: int):
    """Uniform candidate bitstrings and uniforms for a rejection sampler.

    Output 2i of the splitmix64 stream gives candidate i (its top n_qubits
    bits, qubit 0 the most significant) and output 2i+1 its uniform in
    [0, 1) (top 53 bits).  Returns (bitstrings uint8 [count][n_qubits],
    candidate indices int64 [count], uniforms float64 [count]).
    """
    z = splitmix64_stream(seed, 2 * count).reshape(count, 2) if count else np.zeros((0, 2), np.uint64)
    idx = (z[:, 0] >> np.uint64(64 - n_qubits)).astype(np.int64)
    shifts = np.arange(n_qubits - 1, -1, -1, dtype=np.int64)
    bits = ((idx[:, None] >> shifts[None, :]) & 1).astype(np.uint8)
    u = (z[:, 1] >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return bits, idx, u


def ghz_circuit(n: int) -> Circuit:
    """H on qubit 0 followed by the CNOT chain (0,1), (1,2), ..."""
    c = Circuit(n)
    c.append((0,), HADAMARD, "H")
    for q in range(n - 1):
        c.append((q, q + 1), CNOT, "CNOT")
    return c


def product_circuit(n: int, layers: int, seed: int) -> Circuit:
    """Only single-qubit gates: random draws from the Sycamore 1q set, 'layers' per qubit."""
    rng = SplitMix64(seed)
    c = Circuit(n)
    for _ in range(layers):
        for q in range(n):
            k = rng.randint(3)
            c.append((q,), ONE_QUBIT_SET[k], ONE_QUBIT_NAMES[k])
    return c
