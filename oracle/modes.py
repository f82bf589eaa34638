"""Coherent-structure identification from the azimuthal correlation of u_z (Sec. II.C).

Test infrastructure (see the package docstring).

Steps, in the order of Sec. II.C:
1. sample the streamwise velocity on a ring of radius r_0 (= 0.78 R) of one
   cross-section at N_theta equally spaced angles theta_n = 2 pi n / N_theta,
   bilinearly interpolated between the four surrounding cells;
2. take the fluctuation du_z about the ring mean;
3. Eq. (newcorrelation) at Delta r = 0: R_uu(Delta theta_k) =
   <du(theta_0) du(theta_0 + Delta theta_k)>_theta0 / <du^2>_theta0;
4. the power of its discrete Fourier transform (written out as a plain O(N^2) sum);
5. the dominant mode: the largest power over 1 <= m <= 10, the smallest m on a tie.

Readings: the fluctuation is taken about the ring mean, which leaves every m >= 1
coefficient unchanged; the DFT stands in for the FFT (same numbers).
"""
import math

import numpy as np


def bilinear(plane, px, py):
    """Bilinear interpolation of a (ny, nx) field at lattice coordinates (px, py)."""
    i0 = np.floor(px).astype(np.int64)
    j0 = np.floor(py).astype(np.int64)
    fx = px - i0
    fy = py - j0
    return ((1 - fx) * (1 - fy) * plane[j0, i0] + fx * (1 - fy) * plane[j0, i0 + 1]
            + (1 - fx) * fy * plane[j0 + 1, i0] + fx * fy * plane[j0 + 1, i0 + 1])


def ring_samples(plane, xc, yc, r, n_theta):
    theta = 2.0 * math.pi * np.arange(n_theta) / n_theta
    return bilinear(plane, xc + r * np.cos(theta), yc + r * np.sin(theta))


def correlation(u):
    """Eq. (newcorrelation) at Delta r = 0 on one ring, returned for every lag k."""
    du = u - u.mean()
    n = len(du)
    var = np.mean(du * du)
    return np.array([np.mean(du * np.roll(du, -k)) for k in range(n)]) / var


def dft(x):
    """X_m = sum_n x_n exp(-2 pi i m n / N), for m = 0..N-1, as a plain double sum."""
    n = len(x)
    k = np.arange(n)
    return np.array([np.sum(x * np.exp(-2j * math.pi * m * k / n)) for m in range(n)])


def correlation_power(u):
    """|DFT(R_uu)|^2 for every mode m."""
    return np.abs(dft(correlation(u))) ** 2


def dominant_mode(u, m_lo=1, m_hi=10):
    """k*: the mode of largest correlation power in [m_lo, m_hi]; ties go to the smallest."""
    p = correlation_power(u)
    best = m_lo
    for m in range(m_lo, m_hi + 1):
        if p[m] > p[best]:
            best = m
    return best


def energies_from_correlation(u, n_modes):
    """Azimuthal energies E_m = |sum_n u_n e^{-i m theta_n}|^2 / N^2 for m = 0..n_modes,
    rebuilt from the correlation: for m >= 1, DFT(R_uu)_m = |U_m|^2 / sum du^2 (Wiener-
    Khinchin), and E_0 is the squared ring mean."""
    n = len(u)
    du = u - u.mean()
    s = np.sum(du * du)
    F = dft(correlation(u)).real
    E = np.empty(n_modes + 1)
    E[0] = u.mean() ** 2
    E[1:] = F[1:n_modes + 1] * s / n ** 2
    return E


def section_planes(nz, n_sections):
    """z index of each cross-section: z_s = floor(s nz / n_sections)."""
    return [(s * nz) // n_sections for s in range(n_sections)]


def run_modes(run, n_sections, ring_r_over_R, n_theta, n_modes):
    """E[s, j, m] for the current state of an oracle.lbm.Run."""
    _, u = run.moments()
    xc, yc = (run.nx - 1) / 2.0, (run.ny - 1) / 2.0
    out = np.zeros((n_sections, len(ring_r_over_R), n_modes + 1))
    for s, z in enumerate(section_planes(run.nz, n_sections)):
        for j, rr in enumerate(ring_r_over_R):
            samples = ring_samples(u[2, z], xc, yc, rr * run.R, n_theta)
            out[s, j] = energies_from_correlation(samples, n_modes)
    return out
