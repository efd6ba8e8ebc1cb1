"""Uneven circuits in one persistent launch (group API), through the C ABI.

Every member circuit is checked against its own CPU state vector; the
captured CUDA graph must reproduce the direct run exactly.
"""
import numpy as np
import pytest

import oracle
from qxgen import workloads as W

from ._util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qx():
    from paper_2110_09894_gb300 import build
    build.build()
    from paper_2110_09894_gb300 import qx as mod
    return mod


def _members(count, max_n):
    out = []
    for j in range(256):
        n = W.batched_specs()[j][0]
        if n > max_n:
            continue
        w = W.batched_circuit_greedy(j)
        if w.peak_rank <= W.BATCHED_MAX_PEAK_RANK:
            out.append(w)
        if len(out) == count:
            break
    return out


def _group(qx, ws, ctas_per_sm=0):
    import torch
    stream = torch.cuda.Stream()
    cs = [qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings),
                        executor=qx.EXEC_GROUP_MEMBER, stream=stream) for w in ws]
    bits = [torch.from_numpy(w.bitstrings).cuda() for w in ws]
    torch.cuda.synchronize()
    return qx.Group(cs, bits, ctas_per_sm), cs


def test_group_matches_statevectors(qx):
    import torch
    ws = _members(24, 22)
    g, cs = _group(qx, ws)
    g.run()
    torch.cuda.synchronize()
    got = g.amplitudes()
    for w, a in zip(ws, got):
        ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
        assert_parity(a, ref, what=w.name)


def test_group_graph_replay_reproduces_the_run(qx):
    import torch
    ws = _members(12, 20)
    g, cs = _group(qx, ws, ctas_per_sm=1)
    g.run()
    torch.cuda.synchronize()
    direct = g.amplitudes()
    for a in g.d_amps:
        a.zero_()
    g.capture()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(direct, g.amplitudes()):
        assert np.array_equal(a, b)


def test_group_rejects_ordinary_handles(qx):
    import torch
    w = _members(1, 18)[0]
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings))
    with pytest.raises(qx.QXError):
        qx.Group([c], [torch.from_numpy(w.bitstrings).cuda()])
    m = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings),
                      executor=qx.EXEC_GROUP_MEMBER)
    with pytest.raises(qx.QXError):  # a member contracts only through its group
        m.contract(w.bitstrings)


def test_autotuner_picks_and_caches(qx, tmp_path, monkeypatch):
    import torch
    from paper_2110_09894_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    ws = _members(6, 18)
    stream = torch.cuda.Stream()
    cs = [qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings),
                        executor=qx.EXEC_GROUP_MEMBER, stream=stream) for w in ws]
    bits = [torch.from_numpy(w.bitstrings).cuda() for w in ws]
    g, best, times = autotune.tuned_group(cs, bits, candidates=(1, 2))
    assert best in (1, 2) and set(times) == {1, 2}
    g2, best2, _ = autotune.tuned_group(cs, bits, candidates=(1, 2))
    assert best2 == best
    g.run()
    torch.cuda.synchronize()
    for w, a in zip(ws, g.amplitudes()):
        ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
        assert_parity(a, ref)
