"""Pins for the oracle's empirical-supremum rejection sampler (Sec. III-B).

The samples are checked against laws fixed from outside the sampler: the
state-vector oracle's |psi|^2 (chi-square goodness of fit on 10 qubits), the
GHZ law (two outcomes of probability 1/2), and the textbook acceptance rate
1/M of rejection sampling with a bound M that dominates the density ratio.
Planted mistakes in the update of M, in the test and in the probability are
caught by one of these.
"""
import numpy as np
import pytest

import oracle
from oracle import sampler as osp
from qxgen import circuits as C

scipy_stats = pytest.importorskip("scipy.stats")

N_Q = 10


@pytest.fixture(scope="module")
def law10():
    circ = C.random_grid_circuit(2, 5, 12, 2024)
    psi = oracle.statevector(N_Q, C.gates_to_records(circ))
    return (psi.real ** 2 + psi.imag ** 2), psi


def _chi2_pvalue(samples, p, min_expected=5.0):
    """Goodness of fit of integer samples to the law p; bins with a small
    expected count are pooled into one."""
    counts = np.bincount(samples, minlength=len(p)).astype(np.float64)
    exp = p * len(samples)
    big = exp >= min_expected
    obs_b = np.append(counts[big], counts[~big].sum())
    exp_b = np.append(exp[big], exp[~big].sum())
    stat = float(np.sum((obs_b - exp_b) ** 2 / exp_b))
    return float(scipy_stats.chi2.sf(stat, len(obs_b) - 1))


def _draw_and_sample(p, n_q, count, warmup, seed):
    n_cand = int(warmup + count * 1.5 * max(1.0, p.max() * len(p)) + 1000)
    _, idx, u = C.sampler_draws(n_q, n_cand, seed)
    s, used, m = osp.sample_from_law(p, n_q, idx, u, warmup, count)
    assert len(s) == count, "draw more candidates"
    return s, used, m, idx


def test_samples_follow_porter_thomas_law(law10):
    p, _ = law10
    s, used, m, idx = _draw_and_sample(p, N_Q, 40000, 20000, 11)
    assert _chi2_pvalue(s, p) > 1e-4
    # the bound is the empirical supremum over every consumed candidate
    w = p[idx[:used]] * (1 << N_Q)
    assert m == pytest.approx(max(1.0, w.max()), rel=1e-12)
    # after a warm-up that saw every outcome M is sup p N, and rejection
    # sampling then needs M iterations per sample on average
    assert m == pytest.approx(p.max() * (1 << N_Q), rel=1e-12)
    assert (used - 20000) / 40000 == pytest.approx(m, rel=0.03)


def test_ghz_law_two_outcomes():
    n = 4
    psi = oracle.statevector(n, C.gates_to_records(C.ghz_circuit(n)))
    p = psi.real ** 2 + psi.imag ** 2
    s, _, m, _ = _draw_and_sample(p, n, 20000, 200, 5)
    assert set(np.unique(s)) == {0, (1 << n) - 1}
    frac = np.mean(s == 0)
    assert abs(frac - 0.5) < 5 * np.sqrt(0.25 / len(s))
    assert m == pytest.approx(8.0, rel=1e-12)


def test_uniform_law_accepts_everything_after_first():
    # p = 1/N everywhere: w = 1 = M, so U * 1 < 1 always holds
    n = 6
    p = np.full(1 << n, 1.0 / (1 << n))
    _, idx, u = C.sampler_draws(n, 500, 9)
    s, used, m = osp.sample_from_law(p, n, idx, u, 0, 500)
    assert used == 500 and m == pytest.approx(1.0) and np.array_equal(s, idx)


def test_split_run_equals_single_run(law10):
    # carrying M and the remaining warm-up across calls is the same sequential run
    p, psi = law10
    _, idx, u = C.sampler_draws(N_Q, 6000, 21)
    amps = np.stack([psi.real[idx], psi.imag[idx]], axis=1)
    whole, used_w, m_w = osp.esup_run(amps, u, N_Q, 700, 300)
    got, start, m, warm, need = [], 0, 1.0, 700, 300
    for cut in (250, 1100, 1101, 3000, 6000):
        acc, used, m = osp.esup_run(amps[start:cut], u[start:cut], N_Q, warm, need, m)
        got += [start + a for a in acc]
        warm = max(0, warm - used)
        need -= len(acc)
        start += used
        if need == 0:
            break
    assert got == whole and start == used_w and m == m_w


def test_max_out_stops_right_after_last_acceptance(law10):
    p, psi = law10
    _, idx, u = C.sampler_draws(N_Q, 2000, 4)
    amps = np.stack([psi.real[idx], psi.imag[idx]], axis=1)
    acc, used, _ = osp.esup_run(amps, u, N_Q, 0, 7)
    assert len(acc) == 7 and used == acc[-1] + 1
    assert osp.esup_run(amps, u, N_Q, 0, 0) == ([], 0, 1.0)
    assert osp.esup_run(amps[:0], u[:0], N_Q, 0, 5) == ([], 0, 1.0)


# --- planted mistakes: the pins above must catch each one ------------------------------------

def test_planted_frozen_bound_fails_chi_square(law10, monkeypatch):
    p, _ = law10
    monkeypatch.setattr(osp, "_update_sup", lambda m, w: m)
    s, _, _, _ = _draw_and_sample(p, N_Q, 40000, 20000, 11)
    assert _chi2_pvalue(s, p) < 1e-10


def test_planted_test_without_bound_fails_chi_square(law10, monkeypatch):
    p, _ = law10
    monkeypatch.setattr(osp, "_accept", lambda u, m, w: u < w)
    s, _, _, _ = _draw_and_sample(p, N_Q, 40000, 20000, 11)
    assert _chi2_pvalue(s, p) < 1e-10


def test_planted_modulus_for_probability_fails_chi_square(law10, monkeypatch):
    p, _ = law10
    monkeypatch.setattr(osp, "_prob", lambda re, im: float(np.hypot(re, im)) / 8.0)
    s, _, _, _ = _draw_and_sample(p, N_Q, 40000, 20000, 11)
    assert _chi2_pvalue(s, p) < 1e-10


def test_planted_missing_candidate_count_fails_rate(law10, monkeypatch):
    # w = p instead of p N: the law is still right but M stays 1 and the
    # rate pin (M iterations per sample) fails
    p, _ = law10
    monkeypatch.setattr(osp, "_prob", lambda re, im: (re * re + im * im) / (1 << N_Q))
    _, idx, u = C.sampler_draws(N_Q, 200000, 11)
    s, used, m = osp.sample_from_law(p, N_Q, idx, u, 1000, 100)
    assert m == 1.0
    assert (used - 1000) / max(1, len(s)) > 10 * p.max() * (1 << N_Q)
