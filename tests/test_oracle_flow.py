"""Pins of the oracle's time loop against closed-form flows and exact symmetries.

* Hagen-Poiseuille: u_z(r) = g (R^2 - r^2) / (4 nu) in a z-periodic pipe (Sec. II.B
  setup with a constant body force), for the three wall rules; the Bouzidi rule of
  Eqs. (fbc1)-(fbc2) is second order and must beat the staircase.
* Taylor-Green vortex in a periodic box: the amplitude decays as exp(-2 nu k^2 t).
* Equivariance: stepping a mirrored or axis-swapped state equals mirroring or
  swapping the stepped state (catches index, sign and transposition mistakes).
* Mass is conserved exactly by half-way bounce-back; the momentum gained per step
  equals the body force minus what the wall takes.
* The paper's parameter arithmetic (Sec. II.B).
"""
import math
import os

import numpy as np
import pytest

from oracle import lbm as O
from oracle.lattice import C, OPP, W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.txt")


def _poiseuille_error(wall, steps=2000, R=8.0, n=20, g=1e-6, omega=1.25):
    r = O.Run(n, n, 1, omega=omega, R=R, wall=wall, g=(0, 0, g))
    r.init()
    r.step(steps)
    _, u = r.moments()
    nu = O.nu_from_omega(omega)
    xc = (n - 1) / 2.0
    x = np.arange(n) - xc
    r2 = (x[None, :] ** 2 + x[:, None] ** 2)
    m = r.fluid[0]
    uz = u[2, 0][m]
    exact = g * (R * R - r2[m]) / (4 * nu)
    return np.max(np.abs(uz - exact)) / exact.max(), u, r


@pytest.mark.parametrize("wall,tol", [("halfway", 0.06), ("fullway", 0.06), ("bouzidi", 0.01)])
def test_hagen_poiseuille(wall, tol):
    err, u, _ = _poiseuille_error(wall)
    assert err < tol, err
    # no cross-flow in the steady state
    assert np.max(np.abs(u[:2])) < 1e-6 * np.max(np.abs(u[2]))


def test_bouzidi_is_more_accurate_than_staircase():
    e_bz, _, _ = _poiseuille_error("bouzidi")
    e_hw, _, _ = _poiseuille_error("halfway")
    assert e_bz < 0.25 * e_hw


def test_bouzidi_at_half_distance_is_halfway(monkeypatch):
    """Eqs. (fbc1)-(fbc2) at Delta = 1/2 reduce to f_ibar(x_f, t+1) = f*_i(x_f, t)."""
    monkeypatch.setattr(O, "wall_fraction", lambda *a: 0.5)
    rng = np.random.default_rng(3)
    runs = []
    for wall in ("bouzidi", "halfway"):
        r = O.Run(14, 14, 4, omega=1.3, R=5.3, wall=wall, g=(1e-5, 0, 2e-5))
        u0 = 0.02 * rng.standard_normal((3, 4, 14, 14)) if not runs else runs[0][1]
        r.init_fields(np.ones((4, 14, 14)), u0)
        r.step(5)
        runs.append((r, u0))
    a, b = runs[0][0].f, runs[1][0].f
    m = runs[0][0].fluid
    assert np.max(np.abs(a[:, m] - b[:, m])) < 1e-16


def test_halfway_and_fullway_reach_the_same_steady_profile():
    _, ua, _ = _poiseuille_error("halfway")
    _, ub, _ = _poiseuille_error("fullway")
    assert np.max(np.abs(ua - ub)) < 1e-12


def test_taylor_green_decay_rate():
    n, U, omega = 32, 0.01, 1.0
    k = 2 * math.pi / n
    x = np.arange(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.zeros((3, 1, n, n))
    u[0, 0] = U * np.sin(k * X) * np.cos(k * Y)
    u[1, 0] = -U * np.cos(k * X) * np.sin(k * Y)
    r = O.Run(n, n, 1, omega=omega, geometry="box")
    r.init_fields(np.ones((1, n, n)), u)
    basis = np.sin(k * X) * np.cos(k * Y)
    amps = []
    ts = [20, 120]
    for t in ts:
        r.step(t - r.t)
        _, uu = r.moments()
        amps.append(np.sum(uu[0, 0] * basis) / np.sum(basis * basis))
    rate = -math.log(amps[1] / amps[0]) / (ts[1] - ts[0])
    nu = O.nu_from_omega(omega)
    assert abs(rate / (2 * nu * k * k) - 1) < 0.01


def _mirror_x(f):
    """Reflect x -> nx-1-x: population i goes to the direction with c_x negated."""
    perm = [next(j for j in range(27) if C[j, 0] == -C[i, 0] and C[j, 1] == C[i, 1] and C[j, 2] == C[i, 2])
            for i in range(27)]
    out = np.empty_like(f)
    for i in range(27):
        out[perm[i]] = f[i][:, :, ::-1]
    return out


def _swap_xy(f):
    perm = [next(j for j in range(27) if C[j, 0] == C[i, 1] and C[j, 1] == C[i, 0] and C[j, 2] == C[i, 2])
            for i in range(27)]
    out = np.empty_like(f)
    for i in range(27):
        out[perm[i]] = np.swapaxes(f[i], 1, 2)
    return out


@pytest.mark.parametrize("wall", ["halfway", "fullway", "bouzidi"])
@pytest.mark.parametrize("op", [_mirror_x, _swap_xy])
def test_step_is_equivariant_under_pipe_symmetries(wall, op):
    n, nz = 16, 6
    rng = np.random.default_rng(11)
    base = O.Run(n, n, nz, omega=1.4, R=6.2, wall=wall, g=(0, 0, 1e-4))
    u0 = 0.03 * rng.standard_normal((3, nz, n, n))
    base.init_fields(1 + 0.01 * rng.standard_normal((nz, n, n)), u0)
    base.f = base.f + 1e-3 * rng.standard_normal(base.f.shape)   # non-equilibrium parts
    other = O.Run(n, n, nz, omega=1.4, R=6.2, wall=wall, g=(0, 0, 1e-4))
    other.f = op(base.f)
    base.step(3)
    other.step(3)
    m = base.fluid
    diff = other.f - op(base.f)
    assert np.max(np.abs(diff[:, m])) < 1e-15


def test_halfway_conserves_mass_and_balances_momentum():
    n, nz = 14, 5
    rng = np.random.default_rng(12)
    r = O.Run(n, n, nz, omega=1.2, R=5.5, wall="halfway", g=(0, 0, 1e-4))
    r.init_fields(np.ones((nz, n, n)), 0.01 * rng.standard_normal((3, nz, n, n)))
    m = r.fluid
    f0 = r.f.copy()
    r.step(1)
    assert abs(r.f[:, m].sum() - f0[:, m].sum()) < 1e-12
    # momentum change = sum rho g (collision) minus 2 f*_i c_i over wall links
    g = np.zeros((3, nz, n, n))
    g[2] = 1e-4
    from oracle.collision import collide
    fstar = f0.copy()
    fstar[:, m] = collide(f0[:, m], g[:, m], 1.2)
    wall = np.zeros(3)
    for i in range(27):
        dst_fluid = np.roll(m, shift=(-C[i, 2], -C[i, 1], -C[i, 0]), axis=(0, 1, 2))
        links = m & ~dst_fluid
        wall += 2 * C[i] * fstar[i][links].sum()
    j0 = np.einsum("ia,i...->a...", C, f0)[:, m].sum(axis=1)
    j1 = np.einsum("ia,i...->a...", C, r.f)[:, m].sum(axis=1)
    rho0 = f0[:, m].sum(axis=0)
    expect = j0 + np.array([0, 0, 1e-4 * rho0.sum()]) - wall
    assert np.max(np.abs(j1 - expect)) < 1e-14


def test_paper_parameter_arithmetic():
    vals = {}
    with open(GOLD) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, v, tol = line.split()
            vals[k] = (float(v), float(tol))
    R, nu, us = vals["R"][0], vals["nu"][0], vals["u_star"][0]
    p = O.paper_parameters(R, nu, us)
    for key in ("Re_tau", "dx_plus", "T_LET"):
        v, tol = vals[key]
        assert abs(p[key] / v - 1) <= tol, key
    assert abs(vals["nz"][0] / R / vals["L_over_R"][0] - 1) <= vals["L_over_R"][1]
    # u* = sqrt(h R / 2) inverts h = 2 u*^2 / R
    assert abs(O.friction_velocity(p["h"], R) - us) < 1e-15


def test_workload_constants_follow_the_paper_relations():
    from paper_2405_12082_gb300 import workloads as Wk
    for cfg in (Wk.C2, Wk.C3):
        p = O.paper_parameters(cfg["R"], cfg["nu"], cfg["u_star"])
        assert abs(p["Re_tau"] - 181.3) < 1e-9
        assert abs(1.0 / p["tau"] - cfg["omega"]) < 1e-14
        assert abs(p["h"] - cfg["h"]) < 1e-20
        assert abs(0.052 * p["T_LET"] - cfg["period"]) < 1e-9
    assert abs(1.0 / (3 * Wk.C4["nu"] + 0.5) - Wk.C4["omega"]) < 1e-15
    assert abs(1.0 / (3 * Wk.C1["nu"] + 0.5) - Wk.C1["omega"]) < 1e-15
    for mem in Wk.ensemble_members():
        assert abs(O.friction_velocity(mem["h"], mem["R"]) - 0.00388) < 1e-15


@pytest.mark.parametrize("model,equilibrium", [("bgk", "hermite6"), ("bgk", "order2"), ("mrt", "order2")])
def test_taylor_green_decay_rate_of_the_ablation_models(model, equilibrium):
    n, U, omega = 32, 0.01, 1.0
    k = 2 * math.pi / n
    X, Y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    u = np.zeros((3, 1, n, n))
    u[0, 0] = U * np.sin(k * X) * np.cos(k * Y)
    u[1, 0] = -U * np.cos(k * X) * np.sin(k * Y)
    r = O.Run(n, n, 1, omega=omega, geometry="box", model=model, equilibrium=equilibrium)
    r.init_fields(np.ones((1, n, n)), u)
    basis = np.sin(k * X) * np.cos(k * Y)
    amps = []
    for t in (20, 120):
        r.step(t - r.t)
        _, uu = r.moments()
        amps.append(np.sum(uu[0, 0] * basis) / np.sum(basis * basis))
    rate = -math.log(amps[1] / amps[0]) / 100
    assert abs(rate / (2 * O.nu_from_omega(omega) * k * k) - 1) < 0.01


def test_taylor_green_decay_is_set_by_the_shear_rates_alone():
    """With the non-conserved, non-shear moments relaxed at 1.5 instead of 1 (a general
    Lambda), the shear wave still decays at 2 nu k^2 with nu from the shear rate."""
    n, U, omega = 32, 0.01, 1.0
    k = 2 * math.pi / n
    X, Y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    u = np.zeros((3, 1, n, n))
    u[0, 0] = U * np.sin(k * X) * np.cos(k * Y)
    u[1, 0] = -U * np.cos(k * X) * np.sin(k * Y)
    rates = np.full(27, 1.5)
    rates[:4] = 1.0
    rates[4:9] = omega
    r = O.Run(n, n, 1, omega=omega, geometry="box", rates=rates)
    r.init_fields(np.ones((1, n, n)), u)
    basis = np.sin(k * X) * np.cos(k * Y)
    amps = []
    for t in (20, 120):
        r.step(t - r.t)
        _, uu = r.moments()
        amps.append(np.sum(uu[0, 0] * basis) / np.sum(basis * basis))
    rate = -math.log(amps[1] / amps[0]) / 100
    assert abs(rate / (2 * O.nu_from_omega(omega) * k * k) - 1) < 0.01


@pytest.mark.parametrize("R,n", [(7.3, 18), (24.0, 52), (149.5, 300)])
def test_wall_fraction_lands_on_the_circle(R, n):
    """For every in-plane link from a fluid column to a solid one, x + Delta c lies on the
    circle r = R and 0 < Delta <= 1 (the wall crosses the link), Eqs. (fbc1)-(fbc2)."""
    xc = yc = (n - 1) / 2.0
    fluid = O.fluid_mask(n, n, 1, R)[0]
    links = 0
    for y in range(n):
        for x in range(n):
            if not fluid[y, x]:
                continue
            for cy in (-1, 0, 1):
                for cx in (-1, 0, 1):
                    if (cx, cy) == (0, 0) or fluid[(y + cy) % n, (x + cx) % n]:
                        continue
                    px, py = x - xc, y - yc
                    d = O.wall_fraction(px, py, cx, cy, R)
                    assert 0.0 < d <= 1.0 + 1e-12
                    assert abs(math.hypot(px + d * cx, py + d * cy) - R) < 1e-9 * R
                    links += 1
    assert links > 0
