"""Literal FP64 time loop of the pipe-flow LBM: geometry, forces, streaming, statistics.

Test infrastructure (see the package docstring).

The state is a (27, nz, ny, nx) float64 array of populations f_i(x), x fastest,
with cell (i, j, k) at lattice position (x, y, z) = (i, j, k).  One step t -> t+1
(Sec. II.A, Eqs. (collision) and (streaming)):

1. g(x, t): the constant acceleration (0, 0, h) of Sec. II.B, plus the trigger
   force of Eq. (TurbForce) while t < t_end, plus an optional per-cell axial field.
2. Collision of every fluid cell with oracle.collision.collide.
3. Two-buffer pull streaming f_i(x, t+1) = f*_i(x - c_i, t), periodic in every
   direction, with the wall rule chosen by `wall`:
   * "halfway":  if x - c_i is solid, f_i(x, t+1) = f*_ibar(x, t)
                 (the Bouzidi rule of Eqs. (fbc1)-(fbc2) at Delta = 1/2);
   * "fullway":  solid cells do not collide, they reverse their populations,
                 f*_i = f_ibar, and every cell streams;
   * "bouzidi":  Eqs. (fbc1)-(fbc2) with the exact fractional wall distance.

Geometry (reading of Sec. II.B): the pipe axis is at ((nx-1)/2, (ny-1)/2) and a cell
is fluid iff its distance to the axis is strictly less than R; z is periodic.  The
"box" geometry is fluid everywhere and periodic in x, y and z.
"""
import math

import numpy as np

from . import rng
from .collision import collide, collide_model, feq_hermite, feq_order2, macroscopic
from .lattice import C, OPP, W


# ----------------------------------------------------------------------------------
# parameters (Sec. II.B)
# ----------------------------------------------------------------------------------
def friction_velocity(h, R):
    """u* = sqrt(h R / 2) for a pipe driven by the body force rho h (Sec. II.B)."""
    return math.sqrt(h * R / 2.0)


def paper_parameters(R, nu, u_star):
    """Derived quantities of Sec. II.B from R, nu and u*.

    Returns Re_tau = u* R / nu, the grid spacing in wall units dx+ = u* / nu (lattice
    spacing 1 over y* = nu / u*), T_LET = R / u*, the body force h = 2 u*^2 / R and
    tau = nu / c_s^2 + 1/2."""
    return {
        "Re_tau": u_star * R / nu,
        "dx_plus": u_star / nu,
        "T_LET": R / u_star,
        "h": 2.0 * u_star ** 2 / R,
        "tau": 3.0 * nu + 0.5,
    }


def nu_from_omega(omega):
    """Inverse of omega = (nu / c_s^2 + 1/2)^{-1}."""
    return (1.0 / omega - 0.5) / 3.0


# ----------------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------------
def axis(nx, ny):
    return (nx - 1) / 2.0, (ny - 1) / 2.0


def fluid_mask(nx, ny, nz, R, geometry="pipe"):
    """Boolean (nz, ny, nx) mask of fluid cells."""
    if geometry == "box":
        return np.ones((nz, ny, nx), dtype=bool)
    xc, yc = axis(nx, ny)
    x = np.arange(nx)[None, :] - xc
    y = np.arange(ny)[:, None] - yc
    col = x * x + y * y < R * R
    return np.broadcast_to(col[None, :, :], (nz, ny, nx)).copy()


def wall_fraction(px, py, cx, cy, R):
    """Fractional distance Delta in (0, 1] from a fluid point (px, py) (relative to the
    axis) to the circle r = R along the in-plane link (cx, cy) (Sec. II.A, Bouzidi)."""
    a = cx * cx + cy * cy
    b = px * cx + py * cy
    c = px * px + py * py - R * R
    return (-b + math.sqrt(b * b - a * c)) / a


# ----------------------------------------------------------------------------------
# forces (Sec. II.B)
# ----------------------------------------------------------------------------------
class Trigger:
    """The divergence-free trigger force of Eq. (TurbForce), summed over modes.

    Each mode m has azimuthal wavenumber k_theta = m, amplitude A0 * weight_m and an
    azimuthal phase phi_m entering as cos(k_theta theta + phi_m), sin(k_theta theta +
    phi_m).  The paper's single mode is modes=[(2, 1.0, 0.0)].  The force acts for
    t < t_end in the band R - l0 - l <= r <= R - l0."""

    def __init__(self, h, R, L, A0=50.0, kappa=0.5, kz=3, period=2000.0, l0=None, l=None,
                 modes=((2, 1.0, 0.0),), t_end=10 ** 18):
        self.h, self.R, self.L = h, R, L
        self.A0, self.kappa, self.kz, self.period = A0, kappa, kz, period
        self.l0 = 0.2 * R if l0 is None else l0
        self.l = 0.4 * R if l is None else l
        self.modes = list(modes)
        self.t_end = t_end

    def cylindrical(self, r, theta, z, t):
        """(F_r, F_theta, F_z) of Eq. (TurbForce), summed over the modes."""
        h, R, L, l, l0 = self.h, self.R, self.L, self.l, self.l0
        kz, kap = self.kz, self.kappa
        st = math.sin(2.0 * math.pi * t / self.period)
        band = (r >= R - l0 - l) & (r <= R - l0)
        rs = np.where(r > 0, r, 1.0)
        arg = 2.0 * math.pi * (R - r - l0) / l
        zc = np.cos(kz * 2.0 * math.pi * z / L)
        zs = np.sin(kz * 2.0 * math.pi * z / L)
        Fr = np.zeros_like(r)
        Ft = np.zeros_like(r)
        Fz = np.zeros_like(r)
        for k_theta, weight, phase in self.modes:
            A0 = self.A0 * weight
            ang = k_theta * theta + phase
            Fr = Fr - h * kap * A0 * (R / rs) * (kz * l / L) * st * (1.0 - np.cos(arg)) * zc * np.cos(ang)
            Ft = Ft + h * (1.0 - kap) * A0 * (kz / k_theta) * (2.0 * math.pi * R / L) * st * np.sin(arg) * zc * np.sin(ang)
            Fz = Fz - h * A0 * (R / rs) * st * np.sin(arg) * zs * np.cos(ang)
        zero = np.zeros_like(r)
        return (np.where(band, Fr, zero), np.where(band, Ft, zero), np.where(band, Fz, zero))

    def cartesian(self, dx, dy, z, t):
        """Cartesian acceleration of the trigger at axis-relative (dx, dy) and height z."""
        r = np.sqrt(dx * dx + dy * dy)
        theta = np.arctan2(dy, dx)
        Fr, Ft, Fz = self.cylindrical(r, theta, z, t)
        ct, sn = np.cos(theta), np.sin(theta)
        return Fr * ct - Ft * sn, Fr * sn + Ft * ct, Fz


# ----------------------------------------------------------------------------------
# the lattice Boltzmann run
# ----------------------------------------------------------------------------------
class Run:
    """A pipe (or periodic box) simulation, advanced literally step by step."""

    def __init__(self, nx, ny, nz, omega, R=None, geometry="pipe", wall="halfway",
                 g=(0.0, 0.0, 0.0), trigger=None, gz_field=None, model="mrt", equilibrium="hermite6",
                 rates=None):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.R = R if R is not None else 0.0
        self.geometry = geometry
        self.omega = float(omega)
        self.wall = wall
        self.g = np.array(g, dtype=np.float64)
        self.trigger = trigger
        self.gz_field = None if gz_field is None else np.asarray(gz_field, dtype=np.float64)
        self.model, self.equilibrium = model, equilibrium
        self.rates = None if rates is None else np.asarray(rates, dtype=np.float64)
        self.fluid = fluid_mask(nx, ny, nz, self.R, geometry)
        self.t = 0
        self.f = np.broadcast_to(W[:, None, None, None], (27, nz, ny, nx)).copy()
        xc, yc = axis(nx, ny)
        self.dx = np.broadcast_to((np.arange(nx) - xc)[None, None, :], (nz, ny, nx))
        self.dy = np.broadcast_to((np.arange(ny) - yc)[None, :, None], (nz, ny, nx))
        self.zz = np.broadcast_to(np.arange(nz, dtype=np.float64)[:, None, None], (nz, ny, nx))
        self.stats_every = 0
        self.stats = None
        self.stats_count = 0
        if wall == "bouzidi":
            self._bouzidi_links()

    # -- initial state -------------------------------------------------------------
    def initial_velocity(self, profile="rest", noise_amp=0.0, seed=0):
        """u_0(x) on fluid cells: rest, Hagen-Poiseuille, or the mean profile of Sec. II.B
        (U+ = delta+ for delta+ <= 10.8, else ln(delta+)/0.4 + 5), plus seeded noise."""
        u = np.zeros((3, self.nz, self.ny, self.nx))
        r = np.sqrt(self.dx ** 2 + self.dy ** 2)
        gz = self.g[2]
        nu = nu_from_omega(self.omega)
        if profile == "laminar":
            u[2] = gz * (self.R ** 2 - r ** 2) / (4.0 * nu)
        elif profile == "loglaw":
            us = friction_velocity(gz, self.R)
            dplus = (self.R - r) * us / nu
            dp = np.maximum(dplus, 1e-300)
            uplus = np.where(dplus <= 10.8, dplus, np.log(dp) / 0.4 + 5.0)
            u[2] = us * uplus
        elif profile != "rest":
            raise ValueError(profile)
        if noise_amp != 0.0:
            cell = np.arange(self.nx * self.ny * self.nz, dtype=np.uint64).reshape(self.nz, self.ny, self.nx)
            for k in range(3):
                u[k] += noise_amp * rng.normal_at(seed, cell, k)
        u[:, ~self.fluid] = 0.0
        return u

    def init(self, profile="rest", noise_amp=0.0, seed=0):
        """f = f^eq(rho = 1, u_0) on fluid cells, rest weights on solid cells."""
        u = self.initial_velocity(profile, noise_amp, seed)
        self.init_fields(np.ones((self.nz, self.ny, self.nx)), u)

    def init_fields(self, rho, u):
        """f = f^eq(rho, u) (Hermite equilibrium) on fluid cells, rest weights elsewhere."""
        self.f = np.broadcast_to(W[:, None, None, None], (27, self.nz, self.ny, self.nx)).copy()
        m = self.fluid
        feq = feq_hermite if self.equilibrium == "hermite6" else feq_order2
        self.f[:, m] = feq(rho[m], u[:, m])
        self.t = 0

    # -- forces ----------------------------------------------------------------------
    def acceleration(self, t):
        """g(x, t) as a (3, nz, ny, nx) array."""
        g = np.zeros((3, self.nz, self.ny, self.nx))
        g += self.g[:, None, None, None]
        if self.trigger is not None and t < self.trigger.t_end:
            fx, fy, fz = self.trigger.cartesian(self.dx, self.dy, self.zz, t)
            g[0] += fx
            g[1] += fy
            g[2] += fz
        if self.gz_field is not None:
            g[2] += self.gz_field
        return g

    # -- macroscopic fields ------------------------------------------------------------
    def moments(self):
        """rho and the force-shifted velocity at the current time (g evaluated at t)."""
        g = self.acceleration(self.t)
        m = self.fluid
        rho = np.zeros((self.nz, self.ny, self.nx))
        u = np.zeros((3, self.nz, self.ny, self.nx))
        r, uu = macroscopic(self.f[:, m], g[:, m])
        rho[m] = r
        u[:, m] = uu
        return rho, u

    # -- statistics (Sec. III.B point statistics) ---------------------------------------
    def enable_stats(self, every):
        self.stats_every = int(every)
        self.stats = np.zeros((4, self.nz, self.ny, self.nx))
        self.stats_count = 0

    def _accumulate(self, g):
        m = self.fluid
        _, u = macroscopic(self.f[:, m], g[:, m])
        uz = u[2]
        for k in range(4):
            self.stats[k][m] += uz ** (k + 1)
        self.stats_count += 1

    # -- one time step ---------------------------------------------------------------------
    def step(self, n=1):
        for _ in range(n):
            self._step()

    def _step(self):
        t = self.t
        g = self.acceleration(t)
        if self.stats_every and t % self.stats_every == 0:
            self._accumulate(g)
        m = self.fluid
        fstar = self.f.copy()
        if self.model == "mrt" and self.equilibrium == "hermite6" and self.rates is None:
            fstar[:, m] = collide(self.f[:, m], g[:, m], self.omega)
        else:
            fstar[:, m] = collide_model(self.f[:, m], g[:, m], self.omega, self.model, self.equilibrium,
                                        self.rates)
        if self.wall == "fullway":
            solid = ~m
            fstar[:, solid] = self.f[OPP][:, solid]
        new = np.empty_like(self.f)
        for i in range(27):
            cx, cy, cz = (int(v) for v in C[i])
            new[i] = np.roll(fstar[i], shift=(cz, cy, cx), axis=(0, 1, 2))
        if self.wall in ("halfway", "bouzidi") and self.geometry == "pipe":
            for i in range(27):
                cx, cy, cz = (int(v) for v in C[i])
                src_fluid = np.roll(m, shift=(cz, cy, cx), axis=(0, 1, 2))
                links = m & ~src_fluid
                new[i][links] = fstar[OPP[i]][links]
            if self.wall == "bouzidi":
                self._bouzidi_apply(new, fstar)
            keep = ~m
            new[:, keep] = self.f[:, keep]
        self.f = new
        self.t = t + 1

    # -- Bouzidi interpolated bounce-back, Eqs. (fbc1)-(fbc2) ---------------------------------
    def _bouzidi_links(self):
        """For every fluid cell x and wall-pointing direction j (x + c_j solid): Delta."""
        self.blinks = []
        m = self.fluid
        xc, yc = axis(self.nx, self.ny)
        for j in range(27):
            cx, cy, cz = (int(v) for v in C[j])
            nb_fluid = np.roll(m, shift=(-cz, -cy, -cx), axis=(0, 1, 2))
            idx = np.argwhere(m & ~nb_fluid)
            for (k, y, x) in idx:
                delta = wall_fraction(x - xc, y - yc, cx, cy, self.R)
                ff = ((k - cz) % self.nz, (y - cy) % self.ny, (x - cx) % self.nx)
                self.blinks.append((j, k, y, x, delta, bool(m[ff]), ff))

    def _bouzidi_apply(self, new, fstar):
        """Overwrite the half-way values with Eqs. (fbc1)-(fbc2).

        Paper notation: the population f*_j(x_f) heading into the wall returns as
        f_jbar(x_f, t+1); x_ff = x_f - c_j.  Where x_ff is not a fluid cell the Delta < 1/2
        branch has no second point and the half-way value is kept."""
        for (j, k, y, x, d, ff_fluid, ff) in self.blinks:
            jb = OPP[j]
            if d >= 0.5:
                val = fstar[j, k, y, x] / (2.0 * d) + (2.0 * d - 1.0) / (2.0 * d) * fstar[jb, k, y, x]
            elif ff_fluid:
                val = 2.0 * d * fstar[j, k, y, x] + (1.0 - 2.0 * d) * fstar[(j,) + ff]
            else:
                val = fstar[j, k, y, x]
            new[jb, k, y, x] = val


def central_moments(acc, count):
    """Mean, variance, skewness S_3 and flatness S_4 from raw sums sum u^k, k = 1..4
    (Sec. III.B: u_rms = <du^2>^(1/2), S_n = <du^n> / u_rms^n, du = u - <u>_t)."""
    s1, s2, s3, s4 = (a / count for a in acc)
    mean = s1
    var = s2 - mean ** 2
    m3 = s3 - 3 * mean * s2 + 2 * mean ** 3
    m4 = s4 - 4 * mean * s3 + 6 * mean ** 2 * s2 - 3 * mean ** 4
    rms = np.sqrt(np.maximum(var, 0.0))
    with np.errstate(divide="ignore", invalid="ignore"):
        S3 = m3 / rms ** 3
        S4 = m4 / rms ** 4
    return mean, rms, S3, S4
