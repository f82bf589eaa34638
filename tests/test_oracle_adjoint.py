"""Pins of oracle.adjoint: central finite differences of the oracle's own FP64 objective
and the dot-product identity <A v, w> = <v, A^T w> of one linearised step."""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import lbm as O
from paper_2405_12082_gb300 import workloads as Wk

NX = NY = 12
NZ, R, OMEGA, T = 4, 4.5, 1.3, 6


def _setup(seed, gz_base=1e-4):
    gz = Wk.gz_field(NZ, NY, NX, base=gz_base, seed=seed, rel_amp=0.5)
    run = O.Run(NX, NY, NZ, omega=OMEGA, R=R, wall="halfway", g=(0, 0, 1e-5), gz_field=gz)
    u0 = Wk.random_velocity((NZ, NY, NX), seed + 1, 0.01)
    run.init_fields(np.ones((NZ, NY, NX)), u0)
    run.f = run.f + Wk.perturbation(run.f.shape, seed + 2, 1e-4) * run.fluid[None]
    return run, gz


@pytest.mark.parametrize("objective", ["ubulk", "wss"])
def test_adjoint_matches_central_differences(objective):
    run, gz = _setup(31)
    f0 = run.f.copy()
    J, dgz, domega = A.adjoint(run, T, objective)
    cells = Wk.choose_cells(run.fluid, 4, seed=5)
    h = 1e-6
    for c in cells:
        idx = np.unravel_index(c, gz.shape)
        gp, gm = gz.copy(), gz.copy()
        gp[idx] += h
        gm[idx] -= h
        Jp = A.objective_value(NX, NY, NZ, R, OMEGA, (0, 0, 1e-5), gp, f0, T, objective)
        Jm = A.objective_value(NX, NY, NZ, R, OMEGA, (0, 0, 1e-5), gm, f0, T, objective)
        fd = (Jp - Jm) / (2 * h)
        assert abs(dgz[idx] - fd) <= 1e-6 * abs(fd) + 1e-12, (objective, c, dgz[idx], fd)
    h = 1e-6
    Jp = A.objective_value(NX, NY, NZ, R, OMEGA + h, (0, 0, 1e-5), gz, f0, T, objective)
    Jm = A.objective_value(NX, NY, NZ, R, OMEGA - h, (0, 0, 1e-5), gz, f0, T, objective)
    fd = (Jp - Jm) / (2 * h)
    assert abs(domega - fd) <= 1e-6 * abs(fd) + 1e-14, (domega, fd)


def test_dot_product_identity_of_one_step():
    run, _ = _setup(41)
    f = run.f.copy()
    g = run.acceleration(0)
    m = run.fluid
    rng = np.random.default_rng(7)
    v = rng.standard_normal(f.shape) * m[None]
    w = rng.standard_normal(f.shape) * m[None]
    # A v by the complex step through the literal step
    probe = O.Run(NX, NY, NZ, omega=OMEGA, R=R, wall="halfway", g=(0, 0, 1e-5), gz_field=run.gz_field)
    probe.f = f.astype(complex) + 1j * A.H * v
    probe._step()
    Av = probe.f.imag / A.H
    ATw, _, _ = A.step_vjp(run, f, g, w)
    lhs = np.sum(Av[:, m] * w[:, m])
    rhs = np.sum(v[:, m] * ATw[:, m])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
