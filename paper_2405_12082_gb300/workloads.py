"""Seeded synthetic workloads shaped like the paper's pipe flow (Sec. II.B).

This module holds configuration numbers and seeded random draws only; it performs
none of the method's arithmetic and is shared by the CUDA-side tests, the bench
and the oracle-side tests alike.  The derived physical parameters below were
obtained once from the relations of Sec. II.B (u* = sqrt(h R / 2),
Re_tau = u* R / nu, T_LET = R / u*, omega = (3 nu + 1/2)^{-1}) keeping the paper's
friction velocity u* = 0.00388 and Re_tau = 181.3, and are stored here as plain
numbers; tests check them against the oracle's parameter routine.  The ensemble
members derive h = 2 u*^2 / R per radius in ensemble_members (configuration only).

Every pipe sits in a square box of side 2R + 4 with its axis at the box centre.
"""
import math

import numpy as np

SEED = 20240520

# Paper's run (Sec. II.B): 300 x 300 x 600, R = 149.5, nu = 0.0032, u* = 0.00388.
PAPER = dict(nx=300, ny=300, nz=600, R=149.5, nu=0.0032, u_star=0.00388, Re_tau=181.3,
             dx_plus=1.212, T_LET=38531, Re=5329.3, A0=50.0, kappa=0.5, kz=3, k_theta=2,
             period_over_T_LET=0.052, l0_over_R=0.2, l_over_R=0.4)

# Plain laminar pipe, FP64, full-way walls: 20 x 20 x 64, R = 8, g = 1e-6, tau = 0.8.
C1 = dict(name="laminar pipe 20x20x64 R=8 fp64 fullway", nx=20, ny=20, nz=64, R=8.0, precision="f64",
          wall="fullway", nu=0.1, omega=1.25, g=(0.0, 0.0, 1e-6), steps=500)

# Turbulent pipe R = 48 at Re_tau = 181.3 with u* = 0.00388:
#   nu = u* R / Re_tau = 1.02724e-3, tau = 0.5030817, h = 2 u*^2 / R = 6.27267e-7,
#   T_LET = R / u* = 12371.1, trigger period 0.052 T_LET = 643.3, U_b ~ 14.7 u*.
C2 = dict(name="pipe 100x100x480 R=48, Re_tau=181.3 parameters, trigger on (developing flow)", nx=100, ny=100, nz=480, R=48.0, precision="f32",
          wall="halfway", nu=1.0272476558190844e-03, omega=1.9877485398325951, h=6.272666666666667e-07,
          u_star=0.00388, period=643.2989690721649, t_trigger=20000,
          noise=0.0028518, stats_every=100, modes_every=100, n_sections=16,
          r_over_R=(0.78,), n_theta=256, n_modes=32, trigger_modes=[(m, 0.25, 0.0) for m in range(1, 5)])

# Large turbulent pipe R = 96: nu = 2.05449e-3, tau = 0.5061635, h = 3.13633e-7, T_LET = 24742.3.
C3 = dict(C2, name="pipe 196x196x1152 R=96, Re_tau=181.3 parameters, trigger on (developing flow)", nx=196, ny=196, nz=1152, R=96.0,
          nu=2.0544953116381688e-03, omega=1.9756462640779777, h=3.1363333333333336e-07,
          period=1286.5979381443299, n_theta=512)

# The paper's own run (Sec. II.B): 300 x 300 x 600, R = 149.5, nu = 0.0032 (tau = 0.5096),
# u* = 0.00388, h = 2 u*^2 / R = 2.01397e-7, T_LET = R / u* = 38530.9; trigger with
# k_theta = 2, kz = 3, A0 = 50, kappa = 0.5, period 0.052 T_LET = 2003.6, active for the
# first 3 T_LET = 115,592 steps; rings at r0 = 0.78 R with 1024 samples.
C_PAPER = dict(name="paper pipe 300x300x600 R=149.5", nx=300, ny=300, nz=600, R=149.5, precision="f32",
               wall="halfway", nu=0.0032, omega=1.9623233908948192, h=2.0139665551839465e-07,
               u_star=0.00388, period=2003.6082474226803, t_trigger=115592, noise=0.0028518,
               stats_every=100, modes_every=20, n_sections=16, r_over_R=(0.78,), n_theta=1024, n_modes=32,
               trigger_modes=[(2, 1.0, 0.0)])

# Batched ensemble: 16 pipes, R drawn from {16, 20, 24, 32}, length 256, tau = 0.5096.
C4 = dict(name="ensemble 16 pipes R in {16,20,24,32} L=256", n=16, radii=(16, 20, 24, 32), nz=256,
          nu=0.0032, omega=1.9623233908948192, u_star=0.00388, noise=0.0028518, steps=5000, precision="f32",
          wall="halfway")

# Adjoint: 52 x 52 x 256, R = 24, tau = 0.8, per-cell g_z = 1e-6, T = 2000.
C5 = dict(name="adjoint pipe 52x52x256 R=24", nx=52, ny=52, nz=256, R=24.0, nu=0.1, omega=1.25, gz=1e-6,
          T=2000, precision="f32", wall="halfway")


def box_side(R):
    return int(2 * R + 4)


def trigger_dict(h, R, nz, period, modes, t_end, A0=50.0, kappa=0.5, kz=3):
    """Parameters of the trigger force (Eq. (TurbForce)): l0 = 0.2 R, l = 0.4 R."""
    return dict(A0=A0, kappa=kappa, kz=kz, l0=0.2 * R, l=0.4 * R, period=period, h=h, t_end=t_end,
                modes=list(modes))


def ensemble_members(seed=SEED, n=16, radii=(16, 20, 24, 32), u_star=0.00388):
    """Seeded member list: radius drawn uniformly from `radii`, noise seed base + k and
    trigger phase 2 pi k / n for member k; per radius the body force h = 2 u*^2 / R, the
    trigger period 0.052 R / u* and a trigger lasting 3 R / u* steps (configuration)."""
    rng = np.random.default_rng(seed)
    Rs = rng.choice(np.array(radii), size=n)
    out = []
    for k in range(n):
        R = float(Rs[k])
        out.append(dict(R=R, seed=seed + k, phase=2.0 * math.pi * k / n, h=2.0 * u_star ** 2 / R,
                        period=0.052 * R / u_star, t_end=int(3 * R / u_star)))
    return out


def gz_field(nz, ny, nx, base, seed=SEED, rel_amp=0.0, dtype=np.float64):
    """Per-cell axial acceleration: base * (1 + rel_amp * U(-1, 1)), seeded."""
    rng = np.random.default_rng(seed)
    f = base * (1.0 + rel_amp * rng.uniform(-1.0, 1.0, size=(nz, ny, nx)))
    return f.astype(dtype)


def perturbation(shape, seed, amp):
    """Seeded uniform noise in [-amp, amp] of the given shape (float64)."""
    rng = np.random.default_rng(seed)
    return amp * rng.uniform(-1.0, 1.0, size=shape)


def random_velocity(shape, seed, amp):
    """Seeded Gaussian velocity field (3, *shape) with standard deviation amp."""
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((3,) + tuple(shape))


def choose_cells(mask, n, seed):
    """n distinct flat indices of True cells of `mask`, seeded."""
    idx = np.flatnonzero(mask.ravel())
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(idx, size=n, replace=False))
