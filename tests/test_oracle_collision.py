"""Pins of oracle.collision: the equilibrium, the printed moment lists, the MRT update.

Each pin compares the oracle with a fact fixed independently of its code:
* the D3Q27 product form of the Hermite equilibrium (a closed form of the same
  distribution that shares no term-by-term structure with the Hermite sum);
* the printed equilibrium moments (App. A, list after Eq. (omegas)) against M^T f^eq;
* the printed forcing moments against the u-derivative of the printed m^eq
  (Guo forcing: R_k = rho g . grad_u (m_k^eq / rho)), taken by complex step;
* conservation of mass and momentum (Eq. (collision) with Guo forcing adds rho g);
* the printed post-collision shear relations (App. A, list after the m^eq);
* the rest state is a fixed point.
"""
import numpy as np
import pytest

from oracle import collision as K
from oracle.lattice import C, CS2, MT, W


def _rand_state(n, seed, umax=0.15):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * rng.standard_normal(n)
    u = umax * (2 * rng.random((3, n)) - 1)
    return rho, u


def _psi(c, u):
    """1-D factor of the D3Q27 product equilibrium: psi(0,u) = 2/3 - u^2,
    psi(+-1, u) = (u^2 + 1/3 +- u)/2 (moments 1, u, u^2 + cs2 of a 3-point rule)."""
    return np.where(c == 0, 2.0 / 3.0 - u * u, (u * u + 1.0 / 3.0 + c * u) / 2.0)


def test_hermite_equilibrium_equals_product_form():
    rho, u = _rand_state(500, 1)
    feq = K.feq_hermite(rho, u)
    prod = rho[None] * np.prod([_psi(C[:, a][:, None].astype(float), u[a][None]) for a in range(3)], axis=0)
    assert np.max(np.abs(feq - prod)) < 1e-15


def test_equilibrium_at_rest_is_the_weights():
    feq = K.feq_hermite(np.ones(1), np.zeros((3, 1)))
    assert np.max(np.abs(feq[:, 0] - W)) < 1e-16


def test_printed_equilibrium_moments_equal_MT_feq():
    rho, u = _rand_state(500, 2)
    lhs = MT @ K.feq_hermite(rho, u)
    rhs = K.meq_printed(rho, u)
    assert np.max(np.abs(lhs - rhs)) < 2e-15


def test_printed_forcing_moments_are_the_velocity_derivative_of_meq():
    rho, u = _rand_state(400, 3)
    rng = np.random.default_rng(4)
    g = 1e-2 * rng.standard_normal((3, 400))
    h = 1e-30
    d = np.zeros((27, 400))
    for a in range(3):
        uc = u.astype(complex)
        uc[a] += 1j * h
        d += g[a] * (K.meq_printed(rho, uc).imag / h)
    R = K.forcing_printed(rho, u, g)
    assert np.max(np.abs(d - R)) < 1e-16


def test_forcing_moments_are_MT_of_the_velocity_derivative_of_feq():
    """The same identity in population space: (M^T)^{-1} R = g . grad_u f^eq."""
    rho, u = _rand_state(200, 5)
    g = np.array([1e-3, -2e-3, 5e-4])[:, None] * np.ones((3, 200))
    h = 1e-30
    d = np.zeros((27, 200))
    for a in range(3):
        uc = u.astype(complex)
        uc[a] += 1j * h
        d += g[a] * (K.feq_hermite(rho, uc).imag / h)
    assert np.max(np.abs(MT @ d - K.forcing_printed(rho, u, g))) < 1e-16


def test_collision_conserves_mass_and_adds_rho_g_momentum():
    rho, u = _rand_state(300, 6)
    rng = np.random.default_rng(7)
    f = K.feq_hermite(rho, u) + 1e-3 * rng.standard_normal((27, 300))
    g = 1e-4 * rng.standard_normal((3, 300))
    fs = K.collide(f, g, 1.7)
    r0 = f.sum(0)
    assert np.max(np.abs(fs.sum(0) - r0) / r0) < 1e-14
    j0 = C.T @ f
    j1 = C.T @ fs
    assert np.max(np.abs(j1 - (j0 + r0 * g))) < 1e-15


@pytest.mark.parametrize("omega", [0.6, 1.0, 1.25, 1.9877])
def test_printed_post_collision_moments_without_force(omega):
    """Without force: m*_k = m^eq_k for k not in 4..8 and m*_k = (1 - omega) m_k +
    omega m^eq_k for the five shear moments, as printed in App. A."""
    rho, u0 = _rand_state(200, 8)
    rng = np.random.default_rng(9)
    f = K.feq_hermite(rho, u0) + 2e-3 * rng.standard_normal((27, 200))
    g = np.zeros((3, 200))
    fs = K.collide(f, g, omega)
    r = f.sum(0)
    u = (C.T @ f) / r
    m = MT @ f
    ms = MT @ fs
    meq = K.meq_printed(r, u)
    for k in range(27):
        if 4 <= k <= 8:
            expect = (1 - omega) * m[k] + omega * meq[k]
        else:
            expect = meq[k]
        assert np.max(np.abs(ms[k] - expect)) < 1e-14, k
    ux, uy, uz = u
    # the printed shear equilibria rho u_x u_y, ..., rho (u_x^2 - u_z^2)
    assert np.allclose(meq[4], r * ux * uy, atol=1e-16)
    assert np.allclose(meq[7], r * (ux ** 2 - uy ** 2), atol=1e-16)
    assert np.allclose(meq[8], r * (ux ** 2 - uz ** 2), atol=1e-16)


def test_rest_state_is_a_fixed_point():
    f = np.repeat(W[:, None], 10, axis=1)
    fs = K.collide(f, np.zeros((3, 10)), 1.3)
    assert np.max(np.abs(fs - f)) < 1e-16


def test_equilibrium_is_a_fixed_point_without_force():
    rho, u = _rand_state(100, 10)
    f = K.feq_hermite(rho, u)
    fs = K.collide(f, np.zeros((3, 100)), 1.4)
    assert np.max(np.abs(fs - f)) < 1e-15


def test_relaxation_rate_from_viscosity():
    """omega = (nu / cs2 + 1/2)^{-1}: tau = 0.5096 for the paper's nu = 0.0032."""
    assert abs(1.0 / K.omega_from_nu(0.0032) - 0.5096) < 1e-12
    assert abs(CS2 - 1.0 / 3.0) < 1e-17


# ---- ablation models (BGK of Eq. (srt); second-order equilibrium) ----------------------

def test_order2_equilibrium_has_the_maxwellian_moments_to_second_order():
    rho, u = _rand_state(200, 21)
    f = K.feq_order2(rho, u)
    c = C.astype(float)
    assert np.max(np.abs(f.sum(0) - rho)) < 1e-15
    assert np.max(np.abs(c.T @ f - rho * u)) < 1e-15
    for a in range(3):
        for b in range(3):
            expect = rho * (u[a] * u[b] + CS2 * (a == b))
            assert np.max(np.abs((c[:, a] * c[:, b]) @ f - expect)) < 1e-15


def test_guo_forcing_moments():
    """sum F = 0, sum c F = rho g, sum c c F = rho (g u + u g) (Guo et al. 2002)."""
    rho, u = _rand_state(100, 22)
    g = 1e-3 * np.random.default_rng(23).standard_normal((3, 100))
    F = K.guo_order2(rho, u, g)
    c = C.astype(float)
    assert np.max(np.abs(F.sum(0))) < 1e-17
    assert np.max(np.abs(c.T @ F - rho * g)) < 1e-17
    for a in range(3):
        for b in range(3):
            expect = rho * (g[a] * u[b] + u[a] * g[b])
            assert np.max(np.abs((c[:, a] * c[:, b]) @ F - expect)) < 1e-17


@pytest.mark.parametrize("equilibrium", ["hermite6", "order2"])
def test_bgk_in_moment_space_equals_the_population_form(equilibrium):
    """Lambda = omega I in Eq. (m*) is Eq. (srt) plus the forcing term of Eq. (collision):
    f* = f - omega (f - f^eq) + (1 - omega / 2) F."""
    rho, u0 = _rand_state(150, 24)
    rng = np.random.default_rng(25)
    feq_fn = K.feq_hermite if equilibrium == "hermite6" else K.feq_order2
    f = feq_fn(rho, u0) + 1e-3 * rng.standard_normal((27, 150))
    g = 1e-4 * rng.standard_normal((3, 150))
    omega = 1.6
    fs = K.collide_model(f, g, omega, "bgk", equilibrium)
    r, u = K.macroscopic(f, g)
    if equilibrium == "hermite6":
        h = 1e-30
        F = np.zeros_like(f)
        for a in range(3):
            uc = u.astype(complex)
            uc[a] += 1j * h
            F += g[a] * K.feq_hermite(r, uc).imag / h
    else:
        F = K.guo_order2(r, u, g)
    expect = f - omega * (f - feq_fn(r, u)) + (1 - omega / 2) * F
    assert np.max(np.abs(fs - expect)) < 1e-14      # rounding of the FP64 (M^T)^{-1}


def test_mrt_with_hermite6_matches_collide():
    rho, u0 = _rand_state(100, 26)
    f = K.feq_hermite(rho, u0) + 1e-3 * np.random.default_rng(27).standard_normal((27, 100))
    g = 1e-4 * np.ones((3, 100))
    assert np.max(np.abs(K.collide_model(f, g, 1.3) - K.collide(f, g, 1.3))) < 1e-16


# ---- a general diagonal relaxation matrix ------------------------------------------------

def _noneq(seed, equilibrium="hermite6"):
    rho, u0 = _rand_state(120, seed)
    feq_fn = K.feq_hermite if equilibrium == "hermite6" else K.feq_order2
    rng = np.random.default_rng(seed + 1)
    return feq_fn(rho, u0) + 1e-3 * rng.standard_normal((27, 120)), 1e-4 * rng.standard_normal((3, 120))


def test_rates_reproduce_the_paper_matrix_and_bgk():
    f, g = _noneq(31)
    lam = K.relaxation_diag(1.37)
    assert np.max(np.abs(K.collide_model(f, g, 0.0, rates=lam) - K.collide(f, g, 1.37))) < 1e-16
    assert np.max(np.abs(K.collide_model(f, g, 0.0, rates=np.full(27, 1.37))
                         - K.collide_model(f, g, 1.37, "bgk"))) < 1e-16


def test_rates_of_the_conserved_moments_do_not_matter():
    """m_0 = rho and m_1..3 = rho (u - g/2) map to rho and rho (u + g/2) whatever their rate."""
    f, g = _noneq(32)
    lam = np.linspace(0.3, 1.8, 27)
    a = K.collide_model(f, g, 0.0, rates=lam)
    lam2 = lam.copy()
    lam2[:4] = [0.1, 1.9, 0.7, 1.3]
    assert np.max(np.abs(a - K.collide_model(f, g, 0.0, rates=lam2))) < 1e-15
    rho, u = K.macroscopic(f, g)
    c = C.astype(float)
    assert np.max(np.abs(a.sum(0) - rho)) < 1e-14
    assert np.max(np.abs(c.T @ a - rho * (u + 0.5 * g))) < 1e-14


@pytest.mark.parametrize("k", [4, 9, 17, 26])
def test_a_single_rate_acts_on_its_moment_only(k):
    """Changing lambda_k changes m*_k by -(delta lambda)(m_k - m_k^eq + R_k / 2) and leaves
    every other post-collision moment as it was."""
    f, g = _noneq(40 + k)
    lam = K.relaxation_diag(1.2)
    lam2 = lam.copy()
    lam2[k] = 0.6
    d = K.MT @ (K.collide_model(f, g, 0.0, rates=lam2) - K.collide_model(f, g, 0.0, rates=lam))
    rho, u = K.macroscopic(f, g)
    s = (K.MT @ f)[k] - K.meq_printed(rho, u)[k] + 0.5 * K.forcing_printed(rho, u, g)[k]
    others = np.delete(np.arange(27), k)
    assert np.max(np.abs(d[others])) < 1e-14
    assert np.max(np.abs(d[k] - (-(0.6 - lam[k]) * s))) < 1e-14
