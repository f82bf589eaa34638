"""Parity at the full workload sizes, in the launch configuration bench.py times.

The oracle cannot step a 4.8 M-cell pipe in seconds, so at full size it checks outputs
it can compute one by one and properties that hold at any size:
* the R = 48, 100 x 100 x 480 FP32 pipe with the four-mode trigger (bench default):
  the initial state of 400 sampled fluid cells (profile + SplitMix64 noise); one even and
  one odd step of 400 sampled cells recomputed by the oracle from the GPU's own previous
  state (pull streaming, half-way walls, literal collision); the ring energies of all 16
  sections from the GPU state; mass conserved by 100 steps;
* the R = 96, 196 x 196 x 1152 pipe in FP32 and FP64: mass conserved within the rounding
  bound of the format over 50 steps, no non-finite cell;
* the 16-pipe ensemble: two members bit-identical to the same pipes run alone.
"""
import math

import numpy as np
import pytest

from oracle import lbm as O
from oracle import modes as Mo
from oracle.collision import feq_hermite, macroscopic
from paper_2405_12082_gb300 import workloads as Wk

import _sampled as S

pytestmark = pytest.mark.gpu


def _c2(lbm):
    cfg = Wk.C2
    grid = lbm.make_grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"], precision="f32", wall="halfway")
    trig = Wk.trigger_dict(h=cfg["h"], R=cfg["R"], nz=cfg["nz"], period=cfg["period"], modes=cfg["trigger_modes"],
                           t_end=cfg["t_trigger"])
    L = lbm.Lattice(grid, lbm.lbm_relax(cfg["omega"]), lbm.make_force(g=(0.0, 0.0, cfg["h"]), trigger=trig))
    tr = O.Trigger(h=cfg["h"], R=cfg["R"], L=cfg["nz"], period=cfg["period"], modes=cfg["trigger_modes"],
                   t_end=cfg["t_trigger"])
    return cfg, L, tr


def _accel(cfg, tr, z, y, x, t):
    xc, yc = (cfg["nx"] - 1) / 2.0, (cfg["ny"] - 1) / 2.0
    fx, fy, fz = tr.cartesian(x - xc, y - yc, z.astype(float), t)
    return np.array([fx, fy, fz + cfg["h"]])


def _sample(cfg, n, seed):
    fluid = O.fluid_mask(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"])
    cells = Wk.choose_cells(fluid, n, seed)
    return fluid, np.unravel_index(cells, fluid.shape)


@pytest.fixture(scope="module")
def c2_state(lbm_lib):
    cfg, L, tr = _c2(lbm_lib)
    # the launch shapes the bench times: 128 x 8 (even steps) and 128 x 7 (odd steps), 2 planes per thread
    assert (L.info()["variant"], L.info()["variant_odd"]) == (6, 9)
    L.init("loglaw", noise_amp=cfg["noise"], seed=Wk.SEED)
    f0 = L.populations()
    L.step(1)
    f1 = L.populations()
    L.step(1)
    f2 = L.populations()
    yield cfg, L, tr, f0, f1, f2
    L.close()


def test_initial_state_on_sampled_cells(c2_state):
    cfg, L, tr, f0, _, _ = c2_state
    fluid, (z, y, x) = _sample(cfg, 400, 1)
    run = O.Run(cfg["nx"], cfg["ny"], 1, omega=cfg["omega"], R=cfg["R"], g=(0, 0, cfg["h"]))
    xc, yc = (cfg["nx"] - 1) / 2.0, (cfg["ny"] - 1) / 2.0
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    us = O.friction_velocity(cfg["h"], cfg["R"])
    dplus = (cfg["R"] - r) * us / O.nu_from_omega(cfg["omega"])
    uz = us * np.where(dplus <= 10.8, dplus, np.log(np.maximum(dplus, 1e-300)) / 0.4 + 5.0)
    flat = ((z * cfg["ny"] + y) * cfg["nx"] + x).astype(np.uint64)
    from oracle import rng
    u = np.stack([cfg["noise"] * rng.normal_at(Wk.SEED, flat, k) for k in range(3)])
    u[2] += uz
    feq = feq_hermite(np.ones(len(x)), u)
    got = f0[:, z, y, x]
    assert np.max(np.abs(got - feq)) < 2e-8        # FP32 storage of f - w
    del run


@pytest.mark.parametrize("step", [0, 1])
def test_one_step_on_sampled_cells(c2_state, step):
    """Even (t = 0 -> 1) and odd (t = 1 -> 2) AA steps."""
    cfg, L, tr, f0, f1, f2 = c2_state
    fluid, (z, y, x) = _sample(cfg, 400, 2 + step)
    prev, nxt = (f0, f1) if step == 0 else (f1, f2)
    expect = S.one_step(cfg, tr, S.host_fetch(prev), step, fluid, z, y, x)
    got = nxt[:, z, y, x]
    assert np.max(np.abs(got - expect)) < 2e-8


def test_ring_energies_of_all_sections(c2_state, lbm_lib):
    cfg, L, tr, f0, f1, f2 = c2_state
    E = L.modes(n_sections=16, r_over_R=(0.78,), n_theta=256, n_modes=32)
    fluid = O.fluid_mask(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"])
    xc, yc = (cfg["nx"] - 1) / 2.0, (cfg["ny"] - 1) / 2.0
    for s, zp in enumerate(Mo.section_planes(cfg["nz"], 16)):
        f = f2[:, zp][:, fluid[zp]]
        yy, xx = np.nonzero(fluid[zp])
        g = _accel(cfg, tr, np.full(len(xx), zp), yy, xx, 2)
        _, u = macroscopic(f, g)
        plane = np.zeros((cfg["ny"], cfg["nx"]))
        plane[yy, xx] = u[2]
        samples = Mo.ring_samples(plane, xc, yc, 0.78 * cfg["R"], 256)
        Eo = Mo.energies_from_correlation(samples, 32)
        assert abs(E[s, 0, 0] - Eo[0]) <= 1e-6 * Eo[0], s
        assert np.max(np.abs(E[s, 0, 1:] - Eo[1:])) <= 1e-4 * np.max(Eo[1:]), s
        assert int(np.argmax(E[s, 0, 1:11])) == int(np.argmax(Eo[1:11])), s


def _rounding_bound(n_fluid, steps, fmax, eps):
    """Mass is conserved exactly by the collision and the half-way walls; in floating point
    every cell and step rounds 27 stored values of |f - w| <= fmax (half an ulp, eps/2
    relative) and as many sums in the collision: |delta mass| <= 54 (eps/2) fmax per cell
    and step."""
    return n_fluid * steps * 54 * (eps / 2) * fmax


def test_mass_is_conserved_at_full_size(c2_state, lbm_lib):
    cfg, L, tr, f0, f1, f2 = c2_state
    from oracle.lattice import W
    fmax = float(np.max(np.abs(f2 - W[:, None, None, None])))
    m0 = lbm_lib.lbm_reduce(L.ctx)
    L.step(100)
    m1 = lbm_lib.lbm_reduce(L.ctx)
    n_fluid = L.info()["n_fluid"]
    assert abs(m1[0] - m0[0]) < _rounding_bound(n_fluid, 100, fmax, 2.0 ** -23)
    assert m1[4] == 0


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_large_pipe_conserves_mass(lbm_lib, precision):
    """The R = 96, 196 x 196 x 1152 pipe (33.4 M fluid cells) for 50 steps: the mass change
    stays inside the rounding bound of the storage format, and no cell turns non-finite."""
    cfg = Wk.C3
    grid = lbm_lib.make_grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"], precision=precision, wall="halfway")
    trig = Wk.trigger_dict(h=cfg["h"], R=cfg["R"], nz=cfg["nz"], period=cfg["period"], modes=cfg["trigger_modes"],
                           t_end=cfg["t_trigger"])
    L = lbm_lib.Lattice(grid, lbm_lib.lbm_relax(cfg["omega"]), lbm_lib.make_force(g=(0.0, 0.0, cfg["h"]),
                                                                                 trigger=trig))
    L.init("loglaw", noise_amp=cfg["noise"], seed=Wk.SEED)
    m0 = lbm_lib.lbm_reduce(L.ctx)
    L.step(50)
    m1 = lbm_lib.lbm_reduce(L.ctx)
    eps = 2.0 ** -23 if precision == "f32" else 2.0 ** -52
    # |f - w| <= w_0 (|drho| + rho |psi - 1|) stays below 0.05 at these velocities (|u| < 0.1)
    assert abs(m1[0] - m0[0]) < _rounding_bound(L.info()["n_fluid"], 50, 0.05, eps)
    assert m1[4] == 0
    L.close()


def test_ensemble_members_at_full_size(lbm_lib):
    lbm = lbm_lib
    cfg = Wk.C4
    members = Wk.ensemble_members(Wk.SEED, cfg["n"], cfg["radii"], cfg["u_star"])
    grids, relaxes, forces = [], [], []
    for mem in members:
        n = Wk.box_side(mem["R"])
        grids.append(lbm.make_grid(n, n, cfg["nz"], mem["R"], precision="f32", wall="halfway"))
        relaxes.append(lbm.lbm_relax(cfg["omega"]))
        trig = Wk.trigger_dict(h=mem["h"], R=mem["R"], nz=cfg["nz"], period=mem["period"],
                               modes=[(2, 1.0, mem["phase"])], t_end=mem["t_end"])
        forces.append(lbm.make_force(g=(0.0, 0.0, mem["h"]), trigger=trig))
    E = lbm.Lattice(None, None, ensemble=(grids, relaxes, forces))
    lbm.lbm_init(E.ctx, "loglaw", noise_amp=cfg["noise"], seed=Wk.SEED)
    lbm.lbm_set_graph(E.ctx, 100)
    E.step(200)
    for k in (0, 9):
        S = lbm.Lattice(grids[k], relaxes[k], forces[k])
        lbm.lbm_init(S.ctx, "loglaw", noise_amp=cfg["noise"], seed=Wk.SEED + k)
        S.step(200)
        E.select(k)
        assert np.array_equal(E.populations(), S.populations()), k
        S.close()
    E.close()
