"""Empirical-supremum rejection sampler on the GPU vs the oracle (Sec. III-B).

* The rejection-test kernel, fed the oracle's own amplitudes, must take every
  decision the oracle takes, bit for bit: same accepted indices, iterations
  consumed and final bound, over ragged sizes, chunk boundaries, early stops,
  carried-in bounds and special values.
* The whole sampler (contraction + tests) computes its amplitudes itself, so
  a decision may differ from the oracle's only where U*M and w are within the
  amplitude error of each other; every other decision must match.
* The samples follow |psi|^2 (chi-square against the state vector).
"""
import numpy as np
import pytest

import oracle
from oracle import sampler as osp
from qxgen import circuits as C
from qxgen import workloads as W
from qxgen.workloads import make_plan

from ._util import assert_parity

pytestmark = pytest.mark.gpu

BIG = 1 << 40


@pytest.fixture(scope="module")
def qx():
    from paper_2110_09894_gb300 import build
    build.build()
    from paper_2110_09894_gb300 import qx as mod
    return mod


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


@pytest.fixture(scope="module")
def law10():
    circ = C.random_grid_circuit(2, 5, 12, 2024)
    return circ, oracle.statevector(10, C.gates_to_records(circ))


def _amps_of(psi, idx):
    return np.ascontiguousarray(np.stack([psi.real[idx], psi.imag[idx]], axis=1))


def _accept_gpu(qx, torch, amps, u, n_qubits, n_warmup, max_out, m0):
    h = qx.qx_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        n = len(u)
        d_a = torch.from_numpy(np.ascontiguousarray(amps, np.float64).reshape(-1, 2)).cuda()
        d_u = torch.from_numpy(np.ascontiguousarray(u, np.float64)).cuda()
        d_acc = torch.full((max(1, min(max_out, n)),), -1, dtype=torch.int64, device="cuda")
        na, nc, m = qx.qx_esup_accept(h, d_a.data_ptr(), d_u.data_ptr(), n, n_qubits, n_warmup, max_out, m0,
                                      d_acc.data_ptr())
        return d_acc[:na].cpu().numpy().tolist(), nc, m
    finally:
        qx.qx_destroy(h)


def _check_same_or_near_tie(acc_gpu, acc_ref, amps_ref, u, n_qubits, m0, tol):
    """Decisions agree except where U*M and w agree to within tol (relative)."""
    flags_g = np.zeros(len(u), bool)
    flags_r = np.zeros(len(u), bool)
    flags_g[acc_gpu] = True
    flags_r[acc_ref] = True
    bad = np.nonzero(flags_g != flags_r)[0]
    if len(bad) == 0:
        return 0
    w = (amps_ref[:, 0] ** 2 + amps_ref[:, 1] ** 2) * float(2 ** n_qubits)
    m_before = np.maximum(m0, np.concatenate([[m0], np.maximum.accumulate(w)[:-1]]))
    for i in bad:
        assert abs(u[i] * m_before[i] - w[i]) <= tol * max(w[i], u[i] * m_before[i]), f"decision {i} differs"
    return len(bad)


# --- the rejection-test kernel alone: bit-exact ------------------------------------------------

@pytest.mark.parametrize("n_cand,n_warmup,max_out,m0", [
    (1, 0, 5, 1.0), (2, 1, BIG, 1.0), (1007, 100, BIG, 1.0), (8192, 0, BIG, 1.0), (8193, 50, BIG, 2.5),
    (30011, 1000, 777, 1.0), (30011, 0, 1, 1.0), (200003, 20000, BIG, 1.0), (100000, 200000, BIG, 1.0)])
def test_accept_kernel_bit_exact(qx, torch, law10, n_cand, n_warmup, max_out, m0):
    _, psi = law10
    _, idx, u = C.sampler_draws(10, n_cand, 100 + n_cand)
    amps = _amps_of(psi, idx)
    want = osp.esup_run(amps, u, 10, n_warmup, max_out, m0)
    got = _accept_gpu(qx, torch, amps, u, 10, n_warmup, max_out, m0)
    assert got[0] == want[0] and got[1] == want[1] and got[2] == want[2]


def test_accept_kernel_stops_at_and_after_chunk_ends(qx, torch, law10):
    _, psi = law10
    _, idx, u = C.sampler_draws(10, 50000, 77)
    amps = _amps_of(psi, idx)
    every, _, _ = osp.esup_run(amps, u, 10, 0, BIG)
    for boundary in (8192, 16384, 40960):
        k = int(np.searchsorted(every, boundary))  # acceptances before the boundary
        for max_out in (k, k + 1):
            want = osp.esup_run(amps, u, 10, 0, max_out)
            got = _accept_gpu(qx, torch, amps, u, 10, 0, max_out, 1.0)
            assert got == (want[0], want[1], want[2])


def test_accept_kernel_special_values(qx, torch):
    rng = np.random.default_rng(5)
    n = 5000
    amps = rng.normal(size=(n, 2)) * 0.05
    amps[rng.integers(0, n, 40), 0] = np.nan
    amps[rng.integers(0, n, 3), 1] = np.inf
    amps[rng.integers(0, n, 200)] = 0.0
    u = rng.random(n)
    u[rng.integers(0, n, 50)] = 0.0
    for m0 in (1.0, 0.0, 7.5):
        want = osp.esup_run(amps, u, 9, 10, BIG, m0)
        got = _accept_gpu(qx, torch, amps, u, 9, 10, BIG, m0)
        assert got[0] == want[0] and got[1] == want[1]
        assert got[2] == want[2] or (np.isnan(got[2]) and np.isnan(want[2]))


def test_accept_edge_counts(qx, torch):
    h = qx.qx_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        assert qx.qx_esup_accept(h, 0, 0, 0, 10, 0, 5, 3.0, 0) == (0, 0, 3.0)
        d = torch.zeros(8, dtype=torch.float64, device="cuda")
        assert qx.qx_esup_accept(h, d.data_ptr(), d.data_ptr(), 4, 10, 0, 0, 3.0, d.data_ptr()) == (0, 0, 3.0)
        with pytest.raises(qx.QXError):
            qx.qx_esup_accept(h, d.data_ptr(), d.data_ptr(), 4, 63, 0, 1, 1.0, d.data_ptr())
        with pytest.raises(qx.QXError):
            qx.qx_esup_accept(h, d.data_ptr(), d.data_ptr(), -1, 10, 0, 1, 1.0, d.data_ptr())
    finally:
        qx.qx_destroy(h)


# --- contraction + tests ------------------------------------------------------------------------

def _sample_case(qx, torch, c, bits, u, n_warmup, max_out):
    n = len(u)
    d_b = torch.from_numpy(np.ascontiguousarray(bits)).cuda()
    d_u = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    d_a = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    d_acc = torch.full((max(1, min(n, max_out)),), -1, dtype=torch.int64, device="cuda")
    na, nc, m = qx.qx_esup_sample(c.h, d_b.data_ptr(), d_u.data_ptr(), n, n_warmup, max_out, 1.0, d_a.data_ptr(),
                                  d_acc.data_ptr())
    return d_acc[:na].cpu().numpy().tolist(), nc, m, d_a.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_sample_matches_oracle_decisions(qx, torch, prec):
    circ = C.random_grid_circuit(3, 4, 10, 606)
    n = 12
    om = np.zeros(n, np.uint8)
    order, sliced, _, _ = make_plan(circ, om, 3, 9)
    c = qx.Contractor(n, C.gates_to_records(circ), om, order, sliced, 1024, precision=prec)
    psi = oracle.statevector(n, C.gates_to_records(circ))
    bits, idx, u = C.sampler_draws(n, 5000, 31 + prec)
    ref_amps = _amps_of(psi, idx)
    acc_r, used_r, m_r = osp.esup_run(ref_amps, u, n, 300, BIG)
    acc_g, used_g, m_g, amps_g = _sample_case(qx, torch, c, bits, u, 300, BIG)
    assert used_g == used_r == 5000
    assert_parity(amps_g[:, 0] + 1j * amps_g[:, 1], psi[idx])
    assert abs(m_g - m_r) <= 1e-4 * m_r
    assert _check_same_or_near_tie(acc_g, acc_r, ref_amps, u, n, 1.0, 1e-4) <= 2
    # an early stop consumes up to the last acceptance only
    acc_g, used_g, _, _ = _sample_case(qx, torch, c, bits, u, 300, 40)
    acc_r, used_r, _ = osp.esup_run(ref_amps, u, n, 300, 40)
    assert len(acc_g) == 40 and used_g == acc_g[-1] + 1
    if acc_g == acc_r:
        assert used_g == used_r
    c.close()


def test_sample_sliced_workload_full_size(qx, torch):
    # the 20-qubit, 64-slice workload of the benchmark, tensor-core form, a piece size of 256
    w = W.sliced()
    c = qx.Contractor(w.n_qubits, w.gates, w.open_mask, w.order, w.sliced, len(w.bitstrings),
                      precision=qx.QX_PREC_3XTF32)
    psi = oracle.statevector(w.n_qubits, w.gates)
    bits, idx, u = C.sampler_draws(w.n_qubits, 1500, 8)
    ref_amps = _amps_of(psi, idx)
    acc_r, _, m_r = osp.esup_run(ref_amps, u, w.n_qubits, 100, BIG)
    acc_g, used_g, m_g, amps_g = _sample_case(qx, torch, c, bits, u, 100, BIG)
    assert used_g == 1500
    assert_parity(amps_g[:, 0] + 1j * amps_g[:, 1], psi[idx])
    assert abs(m_g - m_r) <= 1e-4 * m_r
    assert _check_same_or_near_tie(acc_g, acc_r, ref_amps, u, w.n_qubits, 1.0, 1e-4) <= 2
    c.close()


def test_sampler_errors_without_plan_or_with_open_qubits(qx, torch):
    circ = C.random_grid_circuit(2, 3, 4, 3)
    om = np.zeros(6, np.uint8)
    om[5] = 1
    order, sliced, _, _ = make_plan(circ, om, 0, 1)
    c = qx.Contractor(6, C.gates_to_records(circ), om, order, sliced, 4)
    d = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(qx.QXError):
        qx.qx_esup_sample(c.h, d.data_ptr(), d.data_ptr(), 4, 0, 4, 1.0, d.data_ptr(), d.data_ptr())
    c.close()


# --- the sampler class -------------------------------------------------------------------------

def _chi2_pvalue(samples, p, min_expected=5.0):
    from scipy import stats
    counts = np.bincount(samples, minlength=len(p)).astype(np.float64)
    exp = p * len(samples)
    big = exp >= min_expected
    obs_b = np.append(counts[big], counts[~big].sum())
    exp_b = np.append(exp[big], exp[~big].sum())
    stat = float(np.sum((obs_b - exp_b) ** 2 / exp_b))
    return float(stats.chi2.sf(stat, len(obs_b) - 1))


def _c10(qx, circ, prec=1, max_bits=4096):
    om = np.zeros(10, np.uint8)
    order, sliced, _, _ = make_plan(circ, om, 2, 4)
    return qx.Contractor(10, C.gates_to_records(circ), om, order, sliced, max_bits, precision=prec)


def test_sampler_class_follows_the_law(qx, law10):
    pytest.importorskip("scipy")
    from paper_2110_09894_gb300.sampler import ESupSampler
    circ, psi = law10
    c = _c10(qx, circ)
    s = ESupSampler(c, seed=3, warmup=20000)
    x = s.sample(20000)
    assert x.shape == (20000, 10)
    code = x.astype(np.int64) @ (1 << np.arange(9, -1, -1))
    p = psi.real ** 2 + psi.imag ** 2
    assert _chi2_pvalue(code, p) > 1e-4
    assert s.m == pytest.approx(p.max() * 1024, rel=1e-4)
    c.close()


def test_sampler_class_is_one_run_across_calls(qx, law10):
    from paper_2110_09894_gb300.sampler import ESupSampler
    circ, psi = law10
    c = _c10(qx, circ, prec=0, max_bits=1000)
    bits, idx, u = C.sampler_draws(10, 60000, 12)

    def stream():
        pos = [0]

        def draw(k):
            a, b = pos[0], pos[0] + k
            pos[0] = b
            return bits[a:b], u[a:b]
        return draw

    split = ESupSampler(c, warmup=2500, batch=1000, draw=stream())
    got = np.concatenate([split.sample(300), split.sample(1), split.sample(450)])
    whole = ESupSampler(c, warmup=2500, batch=1000, draw=stream())
    assert np.array_equal(got, whole.sample(751))
    assert split.iterations == whole.iterations and split.m == whole.m
    # against the oracle over the same stream (a near tie may flip a decision)
    acc_r, used_r, m_r = osp.esup_run(_amps_of(psi, idx), u, 10, 2500, 751)
    assert split.m == pytest.approx(m_r, rel=1e-5)
    if split.iterations == used_r:
        assert np.mean(np.all(got == bits[acc_r], axis=1)) > 0.99
    c.close()
