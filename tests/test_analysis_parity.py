"""The library's host analysis functions (dominant modes, transition matrices, self-mode
correlation) against the oracle on seeded series; exact for counts."""
import numpy as np
import pytest

from oracle import stochastic as St


@pytest.fixture(scope="module")
def series():
    rng = np.random.default_rng(20240520)
    s = rng.integers(0, 13, 5000).astype(np.int32)      # includes values outside 1..10
    s[100:400] = 2                                      # a persistent stretch
    return s


@pytest.mark.parametrize("lag", [1, 2, 5])
def test_transition_matrix_parity(lbm_lib, series, lag):
    T, c = lbm_lib.lbm_transition_matrix(series, 1, 10, lag)
    To, co = St.transition_matrix(series, 1, 10, lag)
    assert np.array_equal(c, co)
    assert np.max(np.abs(T - To)) == 0.0


def test_decimated_series_matrix_equals_pooled_lag_of_one_phase(lbm_lib, series):
    """Lag d pools all d phases of the decimated series; one phase alone is a subset."""
    _, c_all = lbm_lib.lbm_transition_matrix(series, 1, 10, 3)
    total = np.zeros_like(c_all)
    for ph in range(3):
        _, c = St.transition_matrix(St.decimate(series, 3, ph), 1, 10, 1)
        total += c
    assert np.array_equal(total, c_all)


def test_mode_correlation_parity(lbm_lib, series):
    F = lbm_lib.lbm_mode_correlation(series, 1, 10, 40)
    for m in range(1, 11):
        assert np.max(np.abs(F[m - 1] - St.self_mode_correlation(series, m, 40))) < 1e-15


def test_dominant_modes_parity(lbm_lib):
    rng = np.random.default_rng(3)
    E = rng.random((16, 2, 33))
    E[3, 0, 4] = E[3, 0, 7] = 5.0                      # a tie: the smaller mode wins
    k = lbm_lib.lbm_dominant_modes(E, ring=0, m_lo=1, m_hi=10)
    expect = [1 + int(np.argmax(E[s, 0, 1:11])) for s in range(16)]
    assert k.tolist() == expect
    assert k[3] == 4
    with pytest.raises(lbm_lib.LbmError):
        lbm_lib.lbm_dominant_modes(E, ring=2)
