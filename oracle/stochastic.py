"""Stochastic analysis of the dominant-mode series and radial statistics profiles.

Test infrastructure (see the package docstring).

Sec. III.C of the paper: the series S = {k*(t0), k*(t0 + Delta), ...} of dominant
azimuthal modes, its transition matrix (column-stochastic, entry (i, j) = probability
of mode i after mode j), the Chapman-Kolmogorov test (the matrix of the series decimated
by d against the d-th power of the undecimated matrix, compared through eigenvalue
magnitudes) and the self-mode correlation F(t - t') = <V_m(t) V_m(t')> - <V_m>^2 with
V_m(t) = delta(m, k*(t)).  Sec. III.B and its reading: per-cell time moments averaged over
cells in radial bins.
"""
import numpy as np

from .lbm import central_moments


def transition_matrix(series, m_lo=1, m_hi=10, lag=1):
    """Counts of the pairs (k*(t), k*(t + lag)) with both values in [m_lo, m_hi] and the
    column-normalised matrix T[i, j] = P(next = m_lo + i | now = m_lo + j)."""
    K = m_hi - m_lo + 1
    counts = np.zeros((K, K), dtype=np.int64)
    for t in range(len(series) - lag):
        a, b = int(series[t]), int(series[t + lag])
        if m_lo <= a <= m_hi and m_lo <= b <= m_hi:
            counts[b - m_lo, a - m_lo] += 1
    col = counts.sum(axis=0)
    T = np.zeros((K, K))
    for j in range(K):
        if col[j] > 0:
            T[:, j] = counts[:, j] / col[j]
    return T, counts


def decimate(series, d, phase=0):
    """Every d-th element of the series, starting at `phase`."""
    return np.asarray(series)[phase::d]


def ck_eigenvalues(series, d, m_lo=1, m_hi=10):
    """Eigenvalue magnitudes (descending) of the matrix of the d-decimated series and of
    the d-th power of the undecimated matrix."""
    T1, _ = transition_matrix(series, m_lo, m_hi, 1)
    Td, _ = transition_matrix(decimate(series, d), m_lo, m_hi, 1)
    ev_d = np.sort(np.abs(np.linalg.eigvals(Td)))[::-1]
    ev_p = np.sort(np.abs(np.linalg.eigvals(np.linalg.matrix_power(T1, d))))[::-1]
    return ev_d, ev_p


def self_mode_correlation(series, m, max_lag):
    """F_m(tau) for tau = 0..max_lag: the mean of V_m(t) V_m(t + tau) over the available
    pairs minus the squared mean of V_m over the whole series."""
    v = (np.asarray(series) == m).astype(np.float64)
    n = len(v)
    p = v.mean()
    return np.array([np.mean(v[:n - tau] * v[tau:]) - p * p for tau in range(max_lag + 1)])


def radial_profile(acc, count, fluid, nx, ny, nbins, dr):
    """[nbins][6]: bin centre, cells, and the bin averages of the per-cell mean, u_rms, S3
    and S4 (acc: [4][nz][ny][nx] raw sums of u_z^k; fluid: [nz][ny][nx] mask)."""
    mean, rms, S3, S4 = central_moments(acc, count)
    xc, yc = (nx - 1) / 2.0, (ny - 1) / 2.0
    nz = acc.shape[1]
    X = np.broadcast_to((np.arange(nx) - xc)[None, None, :], (nz, ny, nx))
    Y = np.broadcast_to((np.arange(ny) - yc)[None, :, None], (nz, ny, nx))
    b = np.floor(np.sqrt(X * X + Y * Y) / dr).astype(np.int64)
    out = np.zeros((nbins, 6))
    for k in range(nbins):
        sel = fluid & (b == k)
        n = sel.sum()
        out[k, 0] = (k + 0.5) * dr
        out[k, 1] = n
        if n:
            S3s = np.where(rms[sel] > 0, S3[sel], 0.0)
            S4s = np.where(rms[sel] > 0, S4[sel], 0.0)
            out[k, 2:] = [mean[sel].mean(), rms[sel].mean(), S3s.mean(), S4s.mean()]
    return out
