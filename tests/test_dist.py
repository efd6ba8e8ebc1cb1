"""Multi-process slice sharding and FP64 recombination on CPU ranks (gloo).

The ranks' partial sums come from the oracle here (no GPU); what is tested is
the sharding and the exchange: the recombined sum equals the full sum, every
rank gets the same bits, and a rank that dies makes the others fail instead
of returning a partial sum.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2110_09894_gb300.dist import _neumaier_sum, shard_range


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_ranges_cover_every_slice_once():
    for n in (1, 2, 7, 64, 1024):
        for world in (1, 2, 3, 8):
            blocks = [shard_range(n, r, world) for r in range(world)]
            covered = [s for lo, hi in blocks for s in range(lo, hi)]
            assert covered == list(range(n))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1


def test_neumaier_sum_is_exactly_rounded_for_cancelling_parts():
    parts = [np.array([1e16, 1.0]), np.array([1.0, -1e-16]), np.array([-1e16, 1e-16])]
    assert np.array_equal(_neumaier_sum(parts), np.array([1.0, 1.0]))


def _worker(rank, world, port, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import datetime

    import torch.distributed as dist

    from oracle import einsum as oe
    from paper_2110_09894_gb300.dist import combine_partials, shard_range
    from tests._util import grid_case
    from qxgen import circuits as C
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    try:
        circ, om, order, sliced, bits = grid_case(3, 3, 8, 17, n_open=2, n_slice=4, n_bits=3)
        recs = C.gates_to_records(circ)
        lo, hi = shard_range(1 << len(sliced), rank, world)
        part = oe.amplitudes(9, recs, om, order, sliced, bits, slices=range(lo, hi))
        if case == "die" and rank == 1:
            os._exit(3)  # leaves without joining the exchange
        total = combine_partials(part)
        q.put((rank, "ok", total))
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error", repr(e)))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(world, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for p in procs:
        p.join(timeout=120)
    while not q.empty():
        r, status, val = q.get()
        out[r] = (status, val)
    for p in procs:
        if p.is_alive():
            p.kill()
    return out


def test_two_ranks_recombine_to_the_full_sum():
    from oracle import einsum as oe
    from qxgen import circuits as C
    from tests._util import grid_case
    out = _run(2, "ok")
    assert set(out) == {0, 1} and all(v[0] == "ok" for v in out.values())
    circ, om, order, sliced, bits = grid_case(3, 3, 8, 17, n_open=2, n_slice=4, n_bits=3)
    full = oe.amplitudes(9, C.gates_to_records(circ), om, order, sliced, bits)
    assert np.max(np.abs(out[0][1] - full)) < 1e-14
    assert np.array_equal(out[0][1], out[1][1])  # same bits on every rank


def test_a_rank_that_dies_gives_an_error_not_a_partial_sum():
    out = _run(2, "die")
    assert 1 not in out
    assert out[0][0] == "error"
