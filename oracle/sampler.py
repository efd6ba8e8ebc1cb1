"""Oracle: empirical-supremum rejection sampling of output bitstrings.

TEST INFRASTRUCTURE ONLY.  Part of the independent CPU oracle; only the
tests, the smoke check and the CPU-baseline leg of the benchmark use it.

What it computes (Sec. III-B, the low-level challenges; the method is the
empirical supremum rejection sampler of Caffo, Booth and Davison, 2002):

* the target is the output law p(x) = |<x|C|0>|^2 over the N = 2^n
  bitstrings; the proposal is uniform, so the density ratio of candidate x
  is w(x) = p(x) * N;
* each iteration draws a candidate X uniformly and a uniform U in [0, 1);
  X is accepted when U < w(X) / M;
* the bound M starts at 1 and, after every iteration, becomes the larger of
  M and w(X) of that iteration's candidate;
* a warm-up of iterations runs first; their acceptances are discarded, only
  the update of M is kept.

Readings taken where the paper leaves the detail open:

* the test uses the M from before the iteration's own update (the update
  comes "after each iteration");
* the comparison U < w / M is taken as U * M < w in FP64 (one rounded
  product, no division), with p = re*re + im*im rounded term by term;
* a candidate whose w is NaN is never accepted and never raises M;
* a run stops right after its max_out-th accepted candidate, so the
  candidates after it are not consumed and do not touch M.

The random draws (candidates and uniforms) are inputs, made by the seeded
generator of qxgen; this module draws nothing itself.

Parity pins: tests/test_oracle_sampler.py (chi-square goodness of fit of
the samples against the state-vector law |psi|^2 on 10 qubits, the GHZ
law, the acceptance rate 1/M of a converged bound, and planted mistakes in
the update and the test that the chi-square check rejects).
"""
from __future__ import annotations

import numpy as np


def _prob(re: float, im: float) -> float:
    """|a|^2 with each product and the sum rounded separately (FP64)."""
    return re * re + im * im


def _accept(u: float, m: float, w: float) -> bool:
    """The rejection test U < w / M, evaluated as U * M < w."""
    return u * m < w


def _update_sup(m: float, w: float) -> float:
    """Empirical supremum update M = max(M, w); NaN leaves M unchanged."""
    return w if w > m else m


def esup_run(amps, uniforms, n_qubits: int, n_warmup: int, max_out: int, m: float = 1.0):
    """Run the sampler over a fixed sequence of candidates.

    amps: [n][2] float64 amplitudes (re, im) of the candidates, in draw order.
    uniforms: [n] float64 uniforms U, one per candidate.
    n_qubits: N = 2**n_qubits possible candidates.
    n_warmup: the first n_warmup iterations only update M.
    max_out: stop after this many accepted candidates (>= 0).
    m: the bound carried in from earlier iterations (1.0 for a fresh run).

    Returns (accepted candidate indices, iterations consumed, final M).
    """
    amps = np.asarray(amps, dtype=np.float64).reshape(-1, 2)
    uniforms = np.asarray(uniforms, dtype=np.float64).reshape(-1)
    n_total = float(2 ** n_qubits)
    out = []
    if max_out <= 0:
        return out, 0, m
    for i in range(amps.shape[0]):
        w = _prob(float(amps[i, 0]), float(amps[i, 1])) * n_total
        hit = _accept(float(uniforms[i]), m, w)
        m = _update_sup(m, w)
        if i >= n_warmup and hit:
            out.append(i)
            if len(out) == max_out:
                return out, i + 1, m
    return out, amps.shape[0], m


def sample_from_law(prob_of_index, n_qubits: int, cand_index, uniforms, n_warmup: int, count: int):
    """Draw `count` samples, with p(x) taken from a table indexed by x.

    prob_of_index: [2**n_qubits] float64 table p(x) (e.g. |psi|^2 from the
    state-vector oracle); cand_index: candidate x values as integers.
    Returns (sample indices x, iterations consumed, final M).
    """
    p = np.asarray(prob_of_index, dtype=np.float64)
    amps = np.stack([np.sqrt(p[cand_index]), np.zeros(len(cand_index))], axis=1)
    acc, used, m = esup_run(amps, uniforms, n_qubits, n_warmup, count)
    return np.asarray(cand_index)[acc], used, m
