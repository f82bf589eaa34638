"""Pins of oracle.stochastic against hand counts, Markov-chain closed forms and the
Chapman-Kolmogorov identity of a Markov chain (Sec. III.C)."""
import numpy as np
import pytest

from oracle import stochastic as St


def test_transition_matrix_by_hand():
    T, c = St.transition_matrix([1, 2, 2, 1, 3], m_lo=1, m_hi=3)
    # pairs (1->2), (2->2), (2->1), (1->3): column j = origin, row i = destination
    assert c.tolist() == [[0, 1, 0], [1, 1, 0], [1, 0, 0]]
    assert np.allclose(T, [[0, 0.5, 0], [0.5, 0.5, 0], [0.5, 0, 0]])


def _markov(T, n, seed, m_lo=1):
    rng = np.random.default_rng(seed)
    K = T.shape[0]
    s = np.empty(n, dtype=np.int64)
    s[0] = 0
    for t in range(1, n):
        s[t] = rng.choice(K, p=T[:, s[t - 1]])
    return s + m_lo


def _random_T(K, seed, diag=0.6):
    rng = np.random.default_rng(seed)
    A = rng.random((K, K)) + diag * K * np.eye(K)
    return A / A.sum(axis=0, keepdims=True)


def test_transition_matrix_estimates_a_markov_chain():
    T = _random_T(4, 1)
    s = _markov(T, 40000, 2)
    Th, _ = St.transition_matrix(s, 1, 4)
    assert np.allclose(Th.sum(axis=0), 1.0)
    assert np.max(np.abs(Th - T)) < 0.02


def test_chapman_kolmogorov_holds_for_a_markov_chain():
    T = _random_T(3, 5)
    s = _markov(T, 60000, 6)
    for d in (2, 3):
        ev_d, ev_p = St.ck_eigenvalues(s, d, 1, 3)
        assert np.max(np.abs(ev_d - ev_p)) < 0.03
        lam = np.sort(np.abs(np.linalg.eigvals(T)))[::-1] ** d
        assert np.max(np.abs(ev_p - lam)) < 0.03


def test_self_mode_correlation_of_a_two_state_chain():
    """Symmetric two-state chain flipping with probability q: F(tau) = (1 - 2q)^tau / 4."""
    q = 0.1
    T = np.array([[1 - q, q], [q, 1 - q]])
    s = _markov(T, 200000, 7)
    F = St.self_mode_correlation(s, 1, 10)
    expect = 0.25 * (1 - 2 * q) ** np.arange(11)
    assert np.max(np.abs(F - expect)) < 0.01


def test_self_mode_correlation_at_lag_zero_is_p_one_minus_p():
    s = np.random.default_rng(8).integers(1, 6, 1000)
    p = np.mean(s == 3)
    assert abs(St.self_mode_correlation(s, 3, 0)[0] - p * (1 - p)) < 1e-15


def test_radial_profile_of_identical_cells():
    rng = np.random.default_rng(9)
    series = 0.05 + 0.004 * rng.standard_normal(300)
    nz, ny, nx = 2, 12, 12
    acc = np.stack([np.full((nz, ny, nx), np.sum(series ** k)) for k in range(1, 5)])
    fluid = np.ones((nz, ny, nx), dtype=bool)
    out = St.radial_profile(acc, len(series), fluid, nx, ny, 4, 2.0)
    d = series - series.mean()
    for row in out:
        if row[1]:
            assert abs(row[2] - series.mean()) < 1e-14
            assert abs(row[3] - np.sqrt(np.mean(d ** 2))) < 1e-12
            assert abs(row[4] - np.mean(d ** 3) / np.mean(d ** 2) ** 1.5) < 1e-8
    assert out[:, 1].sum() == fluid.sum() - np.sum(
        np.floor(np.sqrt(((np.arange(nx) - 5.5)[None, :] ** 2 + (np.arange(ny) - 5.5)[:, None] ** 2)) / 2.0) >= 4) * nz
