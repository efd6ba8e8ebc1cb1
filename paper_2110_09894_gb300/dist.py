"""Slice sharding across processes (one GPU each) and the FP64 recombination.

Sec. IV-A distributes slices over an MPI sub-communicator and recombines the
partial results.  Here every rank contracts a contiguous block of slices on
its own GPU (``qx_contract_slices``) and the only exchange is an all-gather
of the FP64 partial amplitude vectors (n_amp x 16 bytes), summed on every
rank in rank order with Neumaier compensation, so all ranks hold the same
result and it does not depend on message timing.  A rank that fails or
never arrives makes the collective raise (process-group timeout) instead of
producing a sum with a missing part.
"""
from __future__ import annotations

import numpy as np


def shard_range(n_slices: int, rank: int, world: int):
    """Contiguous block of slices [lo, hi) for `rank` (blocks differ in size by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n_slices, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _neumaier_sum(parts):
    """Compensated sum of a list of float64 arrays, in list order."""
    s = np.zeros_like(parts[0])
    c = np.zeros_like(parts[0])
    for x in parts:
        t = s + x
        big = np.abs(s) >= np.abs(x)
        c += np.where(big, (s - t) + x, (x - t) + s)
        s = t
    return s + c


def combine_partials(partial: np.ndarray, group=None) -> np.ndarray:
    """All-gather complex128 partial sums over the process group and add them in rank order."""
    import torch
    import torch.distributed as dist
    part = np.ascontiguousarray(np.asarray(partial, dtype=np.complex128))
    flat = torch.from_numpy(part.view(np.float64).reshape(-1).copy())
    world = dist.get_world_size(group)
    gathered = [torch.empty_like(flat) for _ in range(world)]
    dist.all_gather(gathered, flat, group=group)
    total = _neumaier_sum([g.numpy() for g in gathered])
    return total.view(np.complex128).reshape(part.shape)


def sharded_amplitudes(contractor, bitstrings, rank: int, world: int, group=None) -> np.ndarray:
    """Amplitudes of all slices: this rank's block on its GPU, then the FP64 recombination."""
    lo, hi = shard_range(contractor.n_slices, rank, world)
    if hi > lo:
        partial = contractor.contract_slices(bitstrings, lo, hi)
    else:
        n = np.asarray(bitstrings).reshape(-1, contractor.n_qubits).shape[0]
        partial = np.zeros((n, 1 << contractor.n_open), dtype=np.complex128)
    return combine_partials(partial, group)

