"""MRT collision with the sixth-order Hermite equilibrium, literally as in Appendix A.

Test infrastructure (see the package docstring).

Every function works on a batch of cells: populations f have shape (27, N), the
density rho shape (N,), velocities and accelerations shape (3, N).

Readings of the text used here (each is listed with its reason in the design notes):
* The force F of Eq. (macroscopic_u) and of the printed R_k is an acceleration g
  (force per unit mass): u = sum_i c_i f_i / rho + g/2, and R_1 = rho g_x.  Only
  under this reading do the printed R_k equal rho g . grad_u (m_k^eq / rho).
* The back transform printed as M^{-1} in Eq. (k*f*) is the inverse of the map
  m = M^T f, i.e. f* = (M^T)^{-1} m*.
* The Hermite polynomials of Eq. (BoltzmannEquilibriumDistribution) are the
  tensor Hermite polynomials of the lattice: per axis H^(1)(c) = c,
  H^(2)(c) = c^2 - c_s^2, and mixed indices take the product over the axes.
"""
import numpy as np

from .lattice import C, CS2, MT, MT_INV, W

CX = C[:, 0].astype(np.float64)[:, None]
CY = C[:, 1].astype(np.float64)[:, None]
CZ = C[:, 2].astype(np.float64)[:, None]


def _h2(c):
    """One-axis second-order Hermite polynomial c^2 - c_s^2."""
    return c * c - CS2


def feq_hermite(rho, u):
    """Eq. (BoltzmannEquilibriumDistribution): f_i^eq, all 27 Hermite terms.

    rho (N,), u (3, N) -> (27, N)."""
    ux, uy, uz = u[0][None, :], u[1][None, :], u[2][None, :]
    cs2, cs4, cs6 = CS2, CS2 ** 2, CS2 ** 3
    cs8, cs10, cs12 = CS2 ** 4, CS2 ** 5, CS2 ** 6
    # second order
    Hxx, Hyy, Hzz = _h2(CX), _h2(CY), _h2(CZ)
    Hxy, Hxz, Hyz = CX * CY, CX * CZ, CY * CZ
    # third order
    Hxxy, Hxxz = Hxx * CY, Hxx * CZ
    Hxyy, Hxzz = CX * Hyy, CX * Hzz
    Hyzz, Hyyz = CY * Hzz, Hyy * CZ
    Hxyz = CX * CY * CZ
    # fourth order
    Hxxyy, Hxxzz, Hyyzz = Hxx * Hyy, Hxx * Hzz, Hyy * Hzz
    Hxyzz, Hxyyz, Hxxyz = CX * CY * Hzz, CX * Hyy * CZ, Hxx * CY * CZ
    # fifth and sixth order
    Hxxyzz, Hxxyyz, Hxyyzz = Hxx * CY * Hzz, Hxx * Hyy * CZ, CX * Hyy * Hzz
    Hxxyyzz = Hxx * Hyy * Hzz

    cu = CX * ux + CY * uy + CZ * uz
    t1 = cu / cs2
    t2 = (Hxx * ux ** 2 + Hyy * uy ** 2 + Hzz * uz ** 2
          + 2.0 * (Hxy * ux * uy + Hxz * ux * uz + Hyz * uy * uz)) / (2.0 * cs4)
    t3 = (Hxxy * ux ** 2 * uy + Hxxz * ux ** 2 * uz + Hxyy * ux * uy ** 2
          + Hxzz * ux * uz ** 2 + Hyzz * uy * uz ** 2 + Hyyz * uy ** 2 * uz
          + 2.0 * Hxyz * ux * uy * uz) / (2.0 * cs6)
    t4 = (Hxxyy * ux ** 2 * uy ** 2 + Hxxzz * ux ** 2 * uz ** 2 + Hyyzz * uy ** 2 * uz ** 2
          + 2.0 * (Hxyzz * ux * uy * uz ** 2 + Hxyyz * ux * uy ** 2 * uz
                   + Hxxyz * ux ** 2 * uy * uz)) / (4.0 * cs8)
    t5 = (Hxxyzz * ux ** 2 * uy * uz ** 2 + Hxxyyz * ux ** 2 * uy ** 2 * uz
          + Hxyyzz * ux * uy ** 2 * uz ** 2) / (4.0 * cs10)
    t6 = Hxxyyzz * ux ** 2 * uy ** 2 * uz ** 2 / (8.0 * cs12)
    return W[:, None] * rho[None, :] * (1.0 + t1 + t2 + t3 + t4 + t5 + t6)


def meq_printed(rho, u):
    """The 27 equilibrium moments m_k^eq as printed after Eq. (omegas). -> (27, N)."""
    ux, uy, uz = u
    x2, y2, z2 = ux * ux, uy * uy, uz * uz
    cs2, cs4, cs6 = CS2, CS2 ** 2, CS2 ** 3
    m = [
        rho,
        rho * ux,
        rho * uy,
        rho * uz,
        rho * ux * uy,
        rho * ux * uz,
        rho * uy * uz,
        rho * (x2 - y2),
        rho * (x2 - z2),
        rho * (x2 + y2 + z2 + 1.0),
        rho * cs2 * ux * (3 * y2 + 3 * z2 + 2),
        rho * cs2 * uy * (3 * x2 + 3 * z2 + 2),
        rho * cs2 * uz * (3 * x2 + 3 * y2 + 2),
        rho * ux * (y2 - z2),
        rho * uy * (x2 - z2),
        rho * uz * (x2 - y2),
        rho * ux * uy * uz,
        rho * cs2 * (3 * (x2 * y2 + x2 * z2 + y2 * z2) + 2 * (x2 + y2 + z2) + 1),
        rho * cs4 * (9 * (x2 * y2 + x2 * z2 - y2 * z2) + 6 * x2 + 1),
        rho * cs2 * (y2 - z2) * (3 * x2 + 1),
        rho * cs2 * uy * uz * (3 * x2 + 1),
        rho * cs2 * ux * uz * (3 * y2 + 1),
        rho * cs2 * ux * uy * (3 * z2 + 1),
        rho * cs4 * ux * (3 * y2 + 1) * (3 * z2 + 1),
        rho * cs4 * uy * (3 * x2 + 1) * (3 * z2 + 1),
        rho * cs4 * uz * (3 * x2 + 1) * (3 * y2 + 1),
        rho * cs6 * (3 * x2 + 1) * (3 * y2 + 1) * (3 * z2 + 1),
    ]
    return np.array(m)


def forcing_printed(rho, u, F):
    """The 27 MRT forcing moments R_k as printed in Appendix A. -> (27, N).

    F is the acceleration g (reading of Eq. (macroscopic_u) noted above)."""
    ux, uy, uz = u
    Fx, Fy, Fz = F
    x2, y2, z2 = ux * ux, uy * uy, uz * uz
    cs2, cs4 = CS2, CS2 ** 2
    zero = np.zeros_like(rho)
    R = [
        zero,
        rho * Fx,
        rho * Fy,
        rho * Fz,
        rho * (Fy * ux + Fx * uy),
        rho * (Fz * ux + Fx * uz),
        rho * (Fz * uy + Fy * uz),
        2 * rho * (Fx * ux - Fy * uy),
        2 * rho * (Fx * ux - Fz * uz),
        2 * rho * (Fx * ux + Fy * uy + Fz * uz),
        cs2 * rho * (6 * ux * (Fy * uy + Fz * uz) + Fx * (2 + 3 * y2 + 3 * z2)),
        cs2 * rho * (6 * uy * (Fx * ux + Fz * uz) + Fy * (2 + 3 * x2 + 3 * z2)),
        cs2 * rho * (6 * uz * (Fx * ux + Fy * uy) + Fz * (2 + 3 * x2 + 3 * y2)),
        rho * (2 * ux * (Fy * uy - Fz * uz) + Fx * (y2 - z2)),
        rho * (2 * uy * (Fx * ux - Fz * uz) + Fy * (x2 - z2)),
        rho * (2 * uz * (Fx * ux - Fy * uy) + Fz * (x2 - y2)),
        rho * (Fx * uy * uz + Fy * ux * uz + Fz * ux * uy),
        2 * cs2 * rho * (Fx * ux * (2 + 3 * y2 + 3 * z2) + Fy * uy * (2 + 3 * x2 + 3 * z2)
                         + Fz * uz * (2 + 3 * x2 + 3 * y2)),
        2 * cs2 * rho * (Fx * ux * (2 + 3 * y2 + 3 * z2) + 3 * Fy * uy * (x2 - z2)
                         + 3 * Fz * uz * (x2 - y2)),
        2 * cs2 * rho * (3 * Fx * ux * (y2 - z2) + (Fy * uy - Fz * uz) * (1 + 3 * x2)),
        cs2 * rho * ((Fz * uy + Fy * uz) * (1 + 3 * x2) + 6 * Fx * ux * uy * uz),
        cs2 * rho * ((Fz * ux + Fx * uz) * (1 + 3 * y2) + 6 * Fy * ux * uy * uz),
        cs2 * rho * ((Fy * ux + Fx * uy) * (1 + 3 * z2) + 6 * Fz * ux * uy * uz),
        cs4 * rho * (Fx * (1 + 3 * y2) * (1 + 3 * z2)
                     + 6 * ux * (Fz * uz * (1 + 3 * y2) + Fy * uy * (1 + 3 * z2))),
        cs4 * rho * (Fy * (1 + 3 * x2) * (1 + 3 * z2)
                     + 6 * uy * (Fz * uz * (1 + 3 * x2) + Fx * ux * (1 + 3 * z2))),
        cs4 * rho * (Fz * (1 + 3 * x2) * (1 + 3 * y2)
                     + 6 * uz * (Fy * uy * (1 + 3 * x2) + Fx * ux * (1 + 3 * y2))),
        2 * cs4 * rho * (Fx * ux * (1 + 3 * y2) * (1 + 3 * z2)
                         + (1 + 3 * x2) * (Fz * uz * (1 + 3 * y2) + Fy * uy * (1 + 3 * z2))),
    ]
    return np.array(R)


def relaxation_diag(omega):
    """Eq. (lambda): Lambda = diag[1,1,1,1, omega x5, 1 x18]."""
    lam = np.ones(27, dtype=np.result_type(omega, np.float64))   # complex omega: complex-step derivatives
    lam[4:9] = omega
    return lam


def omega_from_nu(nu):
    """omega = 1/tau = (nu / c_s^2 + 1/2)^{-1}, stated after Eq. (lambda)."""
    return 1.0 / (nu / CS2 + 0.5)


def macroscopic(f, g):
    """Eqs. (macroscopic_rho), (macroscopic_u): rho = sum f, u = sum c f / rho + g/2."""
    rho = f.sum(axis=0)
    j = C.T.astype(np.float64) @ f
    u = j / rho[None, :] + 0.5 * g
    return rho, u


def feq_order2(rho, u):
    """Second-order truncation of the Maxwell-Boltzmann equilibrium (the 'LBM-O(2)' of
    Sec. III.B's comparison): w rho [1 + c.u / cs2 + (c.u)^2 / (2 cs2^2) - u.u / (2 cs2)]."""
    cu = CX * u[0][None] + CY * u[1][None] + CZ * u[2][None]
    uu = (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)[None]
    return W[:, None] * rho[None, :] * (1.0 + cu / CS2 + cu ** 2 / (2 * CS2 ** 2) - uu / (2 * CS2))


def guo_order2(rho, u, g):
    """Guo et al. (2002) forcing populations for the second-order equilibrium:
    w rho [(c - u) . g / cs2 + (c . u)(c . g) / cs2^2]."""
    cu = CX * u[0][None] + CY * u[1][None] + CZ * u[2][None]
    cg = CX * g[0][None] + CY * g[1][None] + CZ * g[2][None]
    ug = (u[0] * g[0] + u[1] * g[1] + u[2] * g[2])[None]
    return W[:, None] * rho[None, :] * ((cg - ug) / CS2 + cu * cg / CS2 ** 2)


def collide_model(f, g, omega, model="mrt", equilibrium="hermite6", rates=None):
    """Eq. (m*) with a choice of relaxation matrix and equilibrium (ablations).

    model "mrt": Lambda of Eq. (lambda); "bgk": Lambda = omega I, i.e. the single-
    relaxation-time operator of Eq. (srt) with the forcing term of Eq. (collision).
    rates (27 numbers, optional): Lambda = diag(rates) in the moment order of Eq.
    (Mmatrix), overriding model.  equilibrium "hermite6": Eq.
    (BoltzmannEquilibriumDistribution) with the printed m^eq and R_k; "order2": the
    second-order equilibrium with Guo forcing."""
    rho, u = macroscopic(f, g)
    m = MT @ f
    if equilibrium == "hermite6":
        meq = meq_printed(rho, u)
        R = forcing_printed(rho, u, g)
    else:
        meq = MT @ feq_order2(rho, u)
        R = MT @ guo_order2(rho, u, g)
    if rates is not None:
        lam = np.asarray(rates, dtype=np.float64)
    elif model == "mrt":
        lam = relaxation_diag(omega)
    else:
        lam = np.full(27, omega, dtype=np.result_type(omega, 1.0))
    lam = lam[:, None]
    mstar = (1.0 - lam) * m + lam * meq + (1.0 - lam / 2.0) * R
    return MT_INV @ mstar


def collide(f, g, omega):
    """Eq. (collision) in moment space, Eq. (m*), then Eq. (k*f*).

    f (27, N) pre-collision populations, g (3, N) acceleration -> f* (27, N)."""
    rho, u = macroscopic(f, g)
    m = MT @ f
    meq = meq_printed(rho, u)
    R = forcing_printed(rho, u, g)
    lam = relaxation_diag(omega)[:, None]
    mstar = (1.0 - lam) * m + lam * meq + (1.0 - lam / 2.0) * R
    return MT_INV @ mstar
