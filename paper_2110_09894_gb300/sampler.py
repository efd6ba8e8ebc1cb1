"""Output bitstrings of a circuit by empirical-supremum rejection sampling.

Sec. III-B: candidates are drawn uniformly, each one's amplitude comes from
the sliced contraction, and a candidate is kept with probability
min(1, p(x) N / M), where the bound M starts at 1 and grows to the largest
p(x) N seen so far; a warm-up of iterations only sets M.  The contraction
and the rejection tests run in libqx (``qx_esup_sample``); this class only
draws the random numbers, moves them to the GPU and collects the accepted
bitstrings.

The run is one sequential stream of iterations.  A call stops right after
its last acceptance; the candidates of the batch it did not consume keep
their amplitudes on the GPU and the next call tests them first (only the
rejection tests run, no contraction).  The bound and the remaining warm-up
carry over, so ``sample(a)`` followed by ``sample(b)`` gives what one
``sample(a + b)`` would, and no amplitude is computed twice.
"""
from __future__ import annotations

import numpy as np

from . import qx


class ESupSampler:
    """Bitstring sampler over a :class:`qx.Contractor` with every qubit closed.

    draw(count) -> (bitstrings uint8 [count][n_qubits], uniforms float64
    [count]) supplies the random numbers; by default a numpy PCG64 generator
    seeded with ``seed`` draws uniform bits and uniforms in [0, 1).
    ``batch`` candidates go to the GPU per call (default: the contractor's
    bitstring capacity).  ``memo`` switches on qx_set_memo for the
    contractor: the steps that no slice and no output bit touch run once.
    """

    def __init__(self, contractor: qx.Contractor, seed: int = 0, warmup: int = 1000, batch: int | None = None,
                 draw=None, memo: bool = True):
        if contractor.n_open:
            raise ValueError("sampling needs every qubit closed")
        self.c = contractor
        if memo:  # the invariant intermediates are computed once for all batches of candidates
            qx.qx_set_memo(contractor.h, 1)
        self.torch = contractor.torch
        self.n_qubits = contractor.n_qubits
        # one contraction piece per batch, so every candidate of a batch has its amplitude
        self.batch = min(int(batch or contractor.max_bits), contractor.max_bits)
        self.warmup_left = int(warmup)
        self.m = 1.0
        self.iterations = 0
        self.contracted = 0
        if draw is None:
            rng = np.random.Generator(np.random.PCG64(seed))

            def draw(count):
                return (rng.integers(0, 2, size=(count, self.n_qubits), dtype=np.uint8), rng.random(count))
        self._draw = draw
        self._bits = np.zeros((0, self.n_qubits), np.uint8)  # host copy of the current batch
        self._off = 0  # first unconsumed candidate of the current batch
        dev = contractor.device
        self._d_bits = self.torch.empty((self.batch, self.n_qubits), dtype=self.torch.uint8, device=dev)
        self._d_u = self.torch.empty(self.batch, dtype=self.torch.float64, device=dev)
        self._d_amps = self.torch.empty((self.batch, 2), dtype=self.torch.float64, device=dev)
        self._d_acc = self.torch.empty(self.batch, dtype=self.torch.int64, device=dev)

    def sample(self, count: int) -> np.ndarray:
        """The next `count` accepted bitstrings, uint8 [count][n_qubits]."""
        out = []
        need = int(count)
        torch = self.torch
        while need > 0:
            left = len(self._bits) - self._off
            if left > 0:  # amplitudes already on the GPU: tests only
                got, used, self.m = qx.qx_esup_accept(
                    self.c.h, self._d_amps.data_ptr() + 16 * self._off, self._d_u.data_ptr() + 8 * self._off, left,
                    self.n_qubits, self.warmup_left, need, self.m, self._d_acc.data_ptr())
                base = self._off
            else:
                b, u = self._draw(self.batch)
                self._bits = np.ascontiguousarray(b, np.uint8)
                n = len(self._bits)
                with torch.cuda.stream(self.c.stream):
                    self._d_bits[:n].copy_(torch.from_numpy(self._bits))
                    self._d_u[:n].copy_(torch.from_numpy(np.ascontiguousarray(u, np.float64)))
                got, used, self.m = qx.qx_esup_sample(self.c.h, self._d_bits.data_ptr(), self._d_u.data_ptr(), n,
                                                      self.warmup_left, need, self.m, self._d_amps.data_ptr(),
                                                      self._d_acc.data_ptr())
                self.contracted += n
                base = self._off = 0
            if got:
                idx = self._d_acc[:got].cpu().numpy()
                out.append(self._bits[base + idx])
            self._off += used
            self.warmup_left = max(0, self.warmup_left - used)
            self.iterations += used
            need -= got
        return np.concatenate(out) if out else np.zeros((0, self.n_qubits), np.uint8)
