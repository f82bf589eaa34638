"""Reverse mode of the literal FP64 step: gradients of time-averaged pipe objectives.

Test infrastructure (see the package docstring).

The paper has no adjoint; this is the plain mathematics of reverse-mode
differentiation applied to the oracle's own step (oracle.lbm.Run, half-way walls):

    f_{t+1} = S(C(f_t; g, omega)),   C = collision of Appendix A, S = streaming
    J = (1/T) sum_{t=0}^{T-1} [ a(f_t) + b(C(f_t)) ]

with two objectives
    UBULK: a = (1/N) sum_x u_z(x, t) over the N fluid cells, b = 0;
    WSS:   a = 0, b = (1 / (2 pi R nz)) sum over wall links (x + c_i solid) of 2 c_iz f*_i(x)
           (the axial momentum the wall receives during the step).

Backward sweep, t = T-1 .. 0 (lambda_T = 0):
    mu_t     = S^T lambda_{t+1} + db/df*_t
    lambda_t = (dC/df_t)^T mu_t + da/df_t
    dJ/dtheta += (dC/dtheta)^T mu_t + da/dtheta,  theta = g_z(x) per cell, omega.

Every Jacobian is taken by the complex step (f + i h e, imaginary part / h), which
is exact to rounding for the polynomial and rational arithmetic of the collision --
a method independent of the hand-derived transpose of the CUDA kernels.  S^T follows
from the pull rule f_i(x, t+1) = f*_i(x - c_i) (x - c_i fluid) or f*_ibar(x): the
adjoint of f*_i(x) collects lambda_i(x + c_i) if x + c_i is fluid, else lambda_ibar(x).
"""
import math

import numpy as np

from .collision import collide, macroscopic
from .lattice import C, OPP

H = 1e-30


def _fluid_shift(mask, c, sign):
    """mask evaluated at x + sign * c for every x (periodic)."""
    cx, cy, cz = (int(v) for v in c)
    return np.roll(mask, shift=(-sign * cz, -sign * cy, -sign * cx), axis=(0, 1, 2))


def wall_links(fluid):
    """Boolean [27][nz][ny][nx]: fluid x whose neighbour x + c_i is solid."""
    return np.array([fluid & ~_fluid_shift(fluid, C[i], +1) for i in range(27)])


def objective_terms(run, f, g, objective):
    """a(f_t) and b(f*_t) of one time step, and f*_t."""
    m = run.fluid
    N = m.sum()
    fs = f.copy()
    fs[:, m] = collide(f[:, m], g[:, m], run.omega)
    if objective == "ubulk":
        _, u = macroscopic(f[:, m], g[:, m])
        return u[2].sum() / N, 0.0, fs
    links = wall_links(m)
    area = 2.0 * math.pi * run.R * run.nz
    b = sum(2.0 * C[i, 2] * fs[i][links[i]].sum() for i in range(27)) / area
    return 0.0, b, fs


def forward(run, T, objective):
    """Runs T steps from run's state; returns J and the pre-collision states f_0..f_{T-1}."""
    states = []
    J = 0.0
    for _ in range(T):
        g = run.acceleration(run.t)
        a, b, _ = objective_terms(run, run.f, g, objective)
        J += (a + b) / T
        states.append((run.f.copy(), g, run.t))
        run.step(1)
    return J, states


def step_vjp(run, f, g, lam_next, objective=None, T=1):
    """One backward step: from lambda_{t+1} and the pre-collision state f_t (with its
    acceleration g) return lambda_t and the contributions to dJ/dg_z and dJ/domega.
    objective None adds no objective terms (the plain transpose of the step)."""
    m = run.fluid
    N = m.sum()
    links = wall_links(m)
    area = 2.0 * math.pi * run.R * run.nz if run.R else 1.0
    # mu = S^T lambda_{t+1} + db/df*
    mu = np.zeros_like(lam_next)
    for i in range(27):
        nb = _fluid_shift(m, C[i], +1)
        pulled = np.roll(lam_next[i], shift=(-int(C[i, 2]), -int(C[i, 1]), -int(C[i, 0])), axis=(0, 1, 2))
        mu[i] = np.where(nb, pulled, lam_next[OPP[i]])
        if objective == "wss":
            mu[i] += np.where(links[i], 2.0 * C[i, 2] / (T * area), 0.0)
    mu[:, ~m] = 0.0
    fm, gm, mum = f[:, m], g[:, m], mu[:, m]
    # lambda_t = (dC/df)^T mu + da/df, one Jacobian column per population
    lam = np.zeros_like(lam_next)
    lam_m = np.zeros_like(fm)
    for i in range(27):
        fc = fm.astype(complex)
        fc[i] += 1j * H
        dcol = collide(fc, gm, run.omega).imag / H
        lam_m[i] = np.sum(mum * dcol, axis=0)
        if objective == "ubulk":
            _, uc = macroscopic(fc, gm)
            lam_m[i] += uc[2].imag / H / (T * N)
    lam[:, m] = lam_m
    # parameters: g_z(x) and omega
    gc = gm.astype(complex)
    gc[2] += 1j * H
    contrib = np.sum(mum * (collide(fm, gc, run.omega).imag / H), axis=0)
    if objective == "ubulk":
        _, uc = macroscopic(fm, gc)
        contrib += uc[2].imag / H / (T * N)
    dgz = np.zeros(m.shape)
    dgz[m] = contrib
    domega = float(np.sum(mum * (collide(fm, gm, run.omega + 1j * H).imag / H)))
    return lam, dgz, domega


def adjoint(run, T, objective):
    """J, dJ/dg_z (per cell, [nz][ny][nx]) and dJ/domega for T steps from run's state,
    g_z(x) being the per-cell axial acceleration (run.gz_field) on top of the constant
    force.  Leaves run at t + T."""
    J, states = forward(run, T, objective)
    lam = np.zeros((27,) + run.fluid.shape)
    dgz = np.zeros(run.fluid.shape)
    domega = 0.0
    for t in range(T - 1, -1, -1):
        f, g, _ = states[t]
        lam, dg, dw = step_vjp(run, f, g, lam, objective, T)
        dgz += dg
        domega += dw
    return J, dgz, domega


def objective_value(nx, ny, nz, R, omega, g, gz_field, f0, T, objective):
    """J alone for a fresh run from populations f0 (used by finite differences)."""
    from .lbm import Run
    run = Run(nx, ny, nz, omega=omega, R=R, wall="halfway", g=g, gz_field=gz_field)
    run.f = f0.copy()
    J, _ = forward(run, T, objective)
    return J
