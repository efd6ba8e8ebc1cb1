"""Uneven circuits in one captured CUDA graph (needs a GPU).

All 256 circuits of the batched workload, each under its stored plan: the
light ones in the persistent group launch of the C ABI, the heavy ones on the
batched executor in 3xTF32, enqueued on one stream and captured as one graph.
Every member is checked against its complex128 state vector (stored by
tests/golden/make_batched_golden.py, which calls only the oracle); the graph
replay must reproduce the eager run exactly.  Smaller group cases check the
persistent launch on its own and the autotuners.
"""
import json
import os

import numpy as np
import pytest

import oracle
from qxgen import workloads as W

from ._util import assert_parity

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def qx():
    from paper_2110_09894_gb300 import build
    build.build()
    from paper_2110_09894_gb300 import qx as mod
    return mod


def _members(count, max_n, max_peak=18):
    """Light members (persistent-launch sized) of the batched workload with at most max_n qubits."""
    out = []
    for j in range(256):
        n = W.batched_specs()[j][0]
        if n > max_n:
            continue
        w = W.batched_circuit(j)
        if w.peak_rank <= max_peak:
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


def test_all_256_members_in_one_graph_vs_statevectors(qx):
    import torch
    from paper_2110_09894_gb300.batch import UnevenBatch
    from tests.golden.make_batched_golden import case_digest
    with open(os.path.join(HERE, "golden", "batched_statevector.json")) as f:
        recs = {r["j"]: r for r in json.load(f)["circuits"]}
    ws = W.batched_members()
    assert len(ws) == 256 and len(recs) == 256
    b = UnevenBatch(ws, precision=qx.QX_PREC_3XTF32)
    assert b.light and b.heavy  # both kinds of member are in the batch
    b.capture()
    eager = b.amplitudes()
    for a in b.d_amps:
        a.zero_()
    torch.cuda.synchronize()  # the zeros (current stream) land before the replay (the batch's stream) writes
    b.replay()
    torch.cuda.synchronize()
    b.check()
    got = b.amplitudes()
    for w, a, e in zip(ws, got, eager):
        assert np.array_equal(a, e), w.name
        r = recs[w.meta["j"]]
        assert r["digest"] == case_digest(w), f"{w.name}: circuit changed; regenerate the golden file"
        ref = (np.array(r["re"]) + 1j * np.array(r["im"])).reshape(a.shape)
        assert_parity(a, ref, what=w.name)
    b.close()


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
    torch.cuda.synchronize()  # the zeros (current stream) land before the group's stream writes
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


def test_uneven_autotuner_picks_settings_and_caches(qx, tmp_path, monkeypatch):
    """Tile family and slice-batch size of heavy members, persistent grid of light ones: every choice is
    timed, cached, and gives amplitudes within the tolerance of the state vector."""
    import torch
    from paper_2110_09894_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    light = _members(3, 18)
    heavy = [w for w in (W.batched_circuit(j) for j in range(256))
             if w.peak_rank > 18 and w.n_qubits <= 22][:2]
    assert len(heavy) == 2
    ws = light + heavy
    b, choice, ms = autotune.tuned_uneven(ws, precision=qx.QX_PREC_3XTF32, ctas_candidates=(1, 2),
                                          heavy_settings=autotune.HEAVY_SETTINGS[:3], min_share=0.0)
    assert choice["ctas_per_sm"] in (1, 2) and set(ms["light_ctas_per_sm"]) == {"1", "2"}
    assert all(f"heavy{i}" in ms for i in b.heavy)
    b2, choice2, _ = autotune.tuned_uneven(ws, precision=qx.QX_PREC_3XTF32)  # from the cache, no timing
    assert choice2 == choice
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    for w, a in zip(ws, b.amplitudes()):
        ref = oracle.sv_amplitudes(w.n_qubits, w.gates, w.open_mask, w.bitstrings)
        assert_parity(a, ref, what=w.name)
    b.close()
    b2.close()
