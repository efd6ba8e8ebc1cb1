"""The C ABI without a GPU: the library loads, exports every declared entry
point, and its host logic (network build, plan checks, sizing) behaves."""
import ctypes
import os
import re

import numpy as np
import pytest

from qxgen import circuits as C
from qxgen.plan import network_legs, plan_cost
from qxgen.workloads import make_plan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qx():
    from paper_2110_09894_gb300 import build
    build.build()
    from paper_2110_09894_gb300 import qx as mod
    mod.load()
    return mod


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(qx_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(qx):
    lib = ctypes.CDLL(qx.library_path())
    declared = _declared()
    assert declared >= set(qx.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_gate_struct_layout():
    assert C.GATE_DTYPE.itemsize == 272
    assert C.GATE_DTYPE.fields["re"][1] == 16 and C.GATE_DTYPE.fields["im"][1] == 144


def _host_handle(qx, circ, om=None):
    h = qx.qx_create(device=-1)
    qx.qx_build_network(h, circ.n_qubits, C.gates_to_records(circ), om)
    return h


def test_network_counts(qx):
    circ = C.random_grid_circuit(3, 4, 8, 1001)
    om = np.zeros(12, np.uint8)
    om[10:] = 1
    h = _host_handle(qx, circ, om)
    nt, nb = qx.qx_network_info(h)
    assert nt == 12 + len(circ.gates) + 10
    assert nb == 12 + sum(len(g.qubits) for g in circ.gates)
    legs, ne, _ = network_legs(12, [g.qubits for g in circ.gates], om)
    assert (nt, nb) == (len(legs), ne)
    qx.qx_destroy(h)


def test_peak_matches_plan(qx):
    circ = C.random_grid_circuit(4, 5, 12, 2001)
    om = np.zeros(20, np.uint8)
    order, sliced, peak, flops = make_plan(circ, om, 6, 2001 + 700000)
    h = _host_handle(qx, circ, om)
    assert qx.qx_set_plan(h, order, sliced) == 1 << peak
    legs, _, _ = network_legs(20, [g.qubits for g in circ.gates], om)
    assert plan_cost(legs, order, sliced)[0] == peak
    s1 = qx.qx_workspace_size(h, 256, 1)
    s2 = qx.qx_workspace_size(h, 256, 100)
    assert 0 < s1 < s2
    qx.qx_destroy(h)


def test_plan_errors(qx):
    circ = C.random_grid_circuit(2, 3, 4, 7)
    om = np.zeros(6, np.uint8)
    order, sliced, _, _ = make_plan(circ, om, 1, 7)
    h = _host_handle(qx, circ, om)
    with pytest.raises(qx.QXError) as e:
        qx.qx_set_plan(h, order[:-1], sliced)
    assert e.value.code == qx.QX_EINVAL
    bad = [list(p) for p in order]
    bad[3][0] = bad[0][0]  # reuses a consumed id
    with pytest.raises(qx.QXError):
        qx.qx_set_plan(h, bad, sliced)
    legs, ne, _ = network_legs(6, [g.qubits for g in circ.gates], om)
    final = legs[-1][0]  # the final wire of qubit 5
    with pytest.raises(qx.QXError):
        qx.qx_set_plan(h, order, [final])
    with pytest.raises(qx.QXError):
        qx.qx_set_plan(h, order, [ne + 3])
    with pytest.raises(qx.QXError):
        qx.qx_set_plan(h, order, [sliced[0], sliced[0]])
    assert qx.qx_set_plan(h, order, sliced) > 0
    # a host-only handle cannot bind device memory
    with pytest.raises(qx.QXError) as e:
        qx.qx_bind_workspace(h, 0, 1 << 20, 4)
    assert e.value.code == qx.QX_ESTATE
    qx.qx_destroy(h)


def test_plan_result_must_match_open_qubits(qx):
    circ = C.random_grid_circuit(2, 2, 3, 9)
    om = np.zeros(4, np.uint8)
    order, sliced, _, _ = make_plan(circ, om, 0, 9)
    h = qx.qx_create(device=-1)
    om2 = om.copy()
    om2[0] = 1
    qx.qx_build_network(h, 4, C.gates_to_records(circ), om2)
    with pytest.raises(qx.QXError):  # a plan for the closed network does not fit the open one
        qx.qx_set_plan(h, order, sliced)
    qx.qx_destroy(h)


def test_state_errors(qx):
    h = qx.qx_create(device=-1)
    with pytest.raises(qx.QXError) as e:
        qx.qx_network_info(h)
    assert e.value.code == qx.QX_ESTATE
    with pytest.raises(qx.QXError):
        qx.qx_workspace_size(h, 1, 1)
    bad = C.gates_to_records(C.ghz_circuit(3))
    bad[1]["q"][1] = 7
    with pytest.raises(qx.QXError) as e:
        qx.qx_build_network(h, 3, bad)
    assert e.value.code == qx.QX_EINVAL
    qx.qx_destroy(h)


def test_missing_library_fails_loudly(qx, tmp_path):
    with pytest.raises(ImportError):
        qx.load(str(tmp_path / "libqx.so"))


def test_sampler_argument_checks_on_host_only_handle(qx):
    h = qx.qx_create(device=-1)
    # nothing to consume: no device work, bound unchanged
    assert qx.qx_esup_accept(h, 0, 0, 0, 10, 0, 5, 2.5, 0) == (0, 0, 2.5)
    for args in [(0, 0, -1, 10, 0, 5, 1.0, 0), (0, 0, 4, 0, 0, 5, 1.0, 0), (0, 0, 4, 63, 0, 5, 1.0, 0),
                 (0, 0, 4, 10, -2, 5, 1.0, 0), (0, 0, 4, 10, 0, 5, 1.0, 0)]:
        with pytest.raises(qx.QXError) as e:
            qx.qx_esup_accept(h, *args)
        assert e.value.code == qx.QX_EINVAL
    with pytest.raises(qx.QXError) as e:  # no network yet
        qx.qx_esup_sample(h, 0, 0, 4, 0, 5, 1.0, 0, 0)
    assert e.value.code == qx.QX_ESTATE
    qx.qx_build_network(h, 3, C.gates_to_records(C.ghz_circuit(3)), np.array([0, 0, 1], np.uint8))
    with pytest.raises(qx.QXError) as e:  # an open qubit
        qx.qx_esup_sample(h, 0, 0, 4, 0, 5, 1.0, 0, 0)
    assert e.value.code == qx.QX_EINVAL
    qx.qx_destroy(h)


def test_memo_switch_on_host_only_handle(qx):
    h = qx.qx_create(device=-1)
    qx.qx_set_memo(h, 1)
    qx.qx_set_memo(h, 0)
    with pytest.raises(qx.QXError) as e:
        qx.qx_set_memo(h, 2)
    assert e.value.code == qx.QX_EINVAL
    qx.qx_destroy(h)


def test_workspace_grows_with_items_and_holds_the_slice_region(qx):
    from qxgen import workloads as W
    w = W.sliced()
    sizes = {}
    for off in (0, 1):
        h = qx.qx_create(-1, precision=1, no_slice_level=off)
        qx.qx_build_network(h, w.n_qubits, w.gates, w.open_mask)
        qx.qx_set_plan(h, w.order, w.sliced)
        sizes[off] = [qx.qx_workspace_size(h, 256, it) for it in (1, 64, 256, 4096)]
        qx.qx_destroy(h)
    for v in sizes.values():
        assert all(a < b for a, b in zip(v, v[1:]))
    # with the per-slice level, one pair needs its per-pair part and one slice's per-slice part
    assert sizes[0][0] != sizes[1][0]
