"""Pins of the oracle's trigger force, ring analysis, statistics and generator.

* Eq. (TurbForce) is divergence free for any kappa (checked numerically in
  cylindrical and in Cartesian coordinates), vanishes outside its radial band and
  is continuous at the band edges.
* Sec. II.C: a ring carrying cos(m theta) has dominant mode m; the energies rebuilt
  from the correlation R_uu equal |FFT|^2 / N^2 (Wiener-Khinchin, against numpy's
  FFT); the plain DFT equals numpy's FFT; bilinear sampling is exact on bilinear
  fields.
* Sec. III.B: central moments from raw power sums equal two-pass moments; known
  skewness and flatness of the exponential distribution.
* SplitMix64 and Box-Muller: a published output value and normal statistics.
"""
import math

import numpy as np
import pytest

from oracle import lbm as O
from oracle import modes as Mo
from oracle import rng


def _trigger(kappa=0.5, modes=((2, 1.0, 0.0),)):
    return O.Trigger(h=6e-7, R=48.0, L=480.0, A0=50.0, kappa=kappa, kz=3, period=643.3, modes=modes)


@pytest.mark.parametrize("kappa", [0.0, 0.5, 0.8])
@pytest.mark.parametrize("modes", [((2, 1.0, 0.0),), ((1, 0.25, 0.3), (2, 0.25, 1.1), (3, 0.25, 0.0), (4, 0.25, 2.0))])
def test_trigger_is_divergence_free(kappa, modes):
    tr = _trigger(kappa, modes)
    rng_ = np.random.default_rng(5)
    r = rng_.uniform(tr.R - tr.l0 - tr.l + 0.5, tr.R - tr.l0 - 0.5, 50)
    th = rng_.uniform(0, 2 * math.pi, 50)
    z = rng_.uniform(0, 480, 50)
    t = 100.0
    e = 1e-4
    Fr_p = tr.cylindrical(r + e, th, z, t)[0] * (r + e)
    Fr_m = tr.cylindrical(r - e, th, z, t)[0] * (r - e)
    Ft_p = tr.cylindrical(r, th + e, z, t)[1]
    Ft_m = tr.cylindrical(r, th - e, z, t)[1]
    Fz_p = tr.cylindrical(r, th, z + e, t)[2]
    Fz_m = tr.cylindrical(r, th, z - e, t)[2]
    div = (Fr_p - Fr_m) / (2 * e) / r + (Ft_p - Ft_m) / (2 * e) / r + (Fz_p - Fz_m) / (2 * e)
    scale = tr.h * tr.A0 * 2 * math.pi / tr.l
    assert np.max(np.abs(div)) < 1e-7 * scale
    # the same in Cartesian coordinates (checks the polar-to-Cartesian rotation)
    x, y = r * np.cos(th), r * np.sin(th)
    dFx = (tr.cartesian(x + e, y, z, t)[0] - tr.cartesian(x - e, y, z, t)[0]) / (2 * e)
    dFy = (tr.cartesian(x, y + e, z, t)[1] - tr.cartesian(x, y - e, z, t)[1]) / (2 * e)
    dFz = (tr.cartesian(x, y, z + e, t)[2] - tr.cartesian(x, y, z - e, t)[2]) / (2 * e)
    assert np.max(np.abs(dFx + dFy + dFz)) < 1e-7 * scale


def test_trigger_band_and_edges():
    tr = _trigger()
    th = np.full(3, 0.3)
    z = np.full(3, 17.0)
    inside = tr.cylindrical(np.array([20.0, 25.0, 30.0]), th, z, 50.0)
    assert np.all(np.abs(inside[2]) > 0)
    outside = tr.cylindrical(np.array([5.0, 18.0, 40.0]), th, z, 50.0)
    for comp in outside:
        assert np.all(comp == 0)
    lo, hi = tr.R - tr.l0 - tr.l, tr.R - tr.l0
    for edge in (lo, hi):
        vals = tr.cylindrical(np.array([edge]), th[:1], z[:1], 50.0)
        for comp in vals:
            assert abs(comp[0]) < 1e-12 * tr.h * tr.A0
    # sin(2 pi t / T) time factor: zero at t = 0 and t = T/2
    for t in (0.0, tr.period / 2):
        vals = tr.cylindrical(np.array([25.0]), th[:1], z[:1], t)
        assert all(abs(c[0]) < 1e-12 * tr.h * tr.A0 for c in vals)


def test_trigger_single_mode_value_by_hand():
    """F_z at r = 25, theta = 0, z = L/(4 kz) (sin = 1), t = T/4 (sin = 1):
    -h A0 (R/r) sin(2 pi (R - r - l0)/l)."""
    tr = _trigger()
    r = 25.0
    val = tr.cylindrical(np.array([r]), np.array([0.0]), np.array([480.0 / 12]), tr.period / 4)[2][0]
    expect = -tr.h * tr.A0 * (tr.R / r) * math.sin(2 * math.pi * (tr.R - r - tr.l0) / tr.l)
    assert abs(val - expect) < 1e-12 * abs(expect)


def test_dft_matches_fft():
    x = np.random.default_rng(1).standard_normal(64)
    assert np.max(np.abs(Mo.dft(x) - np.fft.fft(x))) < 1e-12


@pytest.mark.parametrize("m", [1, 2, 3, 5, 7, 10])
def test_dominant_mode_of_a_pure_ring(m):
    n = 128
    th = 2 * math.pi * np.arange(n) / n
    rng_ = np.random.default_rng(m)
    u = 0.05 + 0.01 * np.cos(m * th + 0.7) + 0.004 * np.cos((m % 10 + 1) * th) + 1e-4 * rng_.standard_normal(n)
    assert Mo.dominant_mode(u) == m


def test_energies_from_correlation_are_wiener_khinchin():
    n = 64
    u = np.random.default_rng(2).standard_normal(n) + 0.3
    E = Mo.energies_from_correlation(u, 20)
    direct = np.abs(np.fft.fft(u)) ** 2 / n ** 2
    assert np.max(np.abs(E[1:] - direct[1:21])) < 1e-14
    assert abs(E[0] - direct[0]) < 1e-14


def test_bilinear_is_exact_on_bilinear_fields():
    ny, nx = 12, 14
    Y, X = np.mgrid[0:ny, 0:nx].astype(float)
    plane = 0.3 + 0.02 * X - 0.05 * Y + 0.001 * X * Y
    rng_ = np.random.default_rng(3)
    px = rng_.uniform(0, nx - 1.01, 40)
    py = rng_.uniform(0, ny - 1.01, 40)
    exact = 0.3 + 0.02 * px - 0.05 * py + 0.001 * px * py
    assert np.max(np.abs(Mo.bilinear(plane, px, py) - exact)) < 1e-14


def test_ring_samples_on_a_linear_field():
    ny = nx = 20
    Y, X = np.mgrid[0:ny, 0:nx].astype(float)
    plane = X.copy()
    s = Mo.ring_samples(plane, 9.5, 9.5, 6.24, 32)
    th = 2 * math.pi * np.arange(32) / 32
    assert np.max(np.abs(s - (9.5 + 6.24 * np.cos(th)))) < 1e-13


def test_central_moments_from_raw_sums_equal_two_pass():
    rng_ = np.random.default_rng(4)
    x = 0.06 + 0.006 * rng_.standard_normal(20000)
    acc = [np.sum(x ** k) for k in range(1, 5)]
    mean, rms, S3, S4 = O.central_moments(np.array(acc), len(x))
    d = x - x.mean()
    assert abs(mean - x.mean()) < 1e-15
    assert abs(rms - np.sqrt(np.mean(d ** 2))) < 1e-12 * rms
    assert abs(S3 - np.mean(d ** 3) / np.mean(d ** 2) ** 1.5) < 1e-8
    assert abs(S4 - np.mean(d ** 4) / np.mean(d ** 2) ** 2) < 1e-8


def test_central_moments_of_exponential():
    x = np.random.default_rng(5).exponential(1.0, 400000)
    acc = np.array([np.sum(x ** k) for k in range(1, 5)])
    mean, rms, S3, S4 = O.central_moments(acc, len(x))
    assert abs(S3 - 2.0) < 0.1
    assert abs(S4 - 9.0) < 0.8


def test_splitmix64_published_first_output():
    """SplitMix64 seeded with 0: first output 0xE220A8397B1DCDAF."""
    assert int(rng.splitmix64_at(0, 0)) == 0xE220A8397B1DCDAF


def test_splitmix64_counter_equals_sequential_state():
    seed = 12345
    state = seed
    for n in range(5):
        state = (state + 0x9E3779B97F4A7C15) % 2 ** 64
        assert int(rng.mix64(np.uint64(state))) == int(rng.splitmix64_at(seed, n))


def test_box_muller_normals():
    z = rng.normal_at(777, np.arange(100000, dtype=np.uint64), 1)
    assert abs(z.mean()) < 0.015
    assert abs(z.var() - 1) < 0.02
    assert abs(np.mean(z ** 4) - 3) < 0.1
    z2 = rng.normal_at(777, np.arange(100000, dtype=np.uint64), 2)
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.015
