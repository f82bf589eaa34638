"""GPU parity of the ablation collision models against the oracle's literal forms.

The models: the single-relaxation-time operator of Eq. (srt) with the forcing term of
Eq. (collision) (Lambda = omega I in Eq. (m*)), and the second-order equilibrium of the
"LBM-O(2)" comparison of Sec. III.B with the forcing g . grad_u f^eq, each alone and
combined.  The oracle runs them in moment space through the 27 x 27 transforms; the
kernels use closed forms, so FP64 results agree to rounding (1e-13 relative after a few
steps, as for the default model).
"""
import numpy as np
import pytest

from _pairs import TRIG_MODES, make_pair, perturbed_state, rel_err

pytestmark = pytest.mark.gpu

MODELS = [("bgk", "hermite6"), ("mrt", "order2"), ("bgk", "order2")]


@pytest.mark.parametrize("model,equilibrium", MODELS)
@pytest.mark.parametrize("wall", ["halfway", "fullway", "bouzidi"])
def test_step_parity(lbm_lib, model, equilibrium, wall):
    """Both AA parities, every wall rule, a ragged 23x19x7 pipe, trigger force on."""
    L, ref = make_pair(lbm_lib, 23, 19, 7, 7.3, precision="f64", wall=wall, omega=1.7, g=(2e-5, -1e-5, 3e-5),
                       trigger=dict(h=1e-4, period=20.0, modes=TRIG_MODES, t_end=100),
                       model=model, equilibrium=equilibrium)
    f0 = perturbed_state(ref, 111)
    L.set_populations(f0)
    for n in (1, 2, 3):
        L.step(n)
        ref.step(n)
        assert rel_err(L.populations(), ref.f, ref.fluid) < 1e-13, n
    L.close()


@pytest.mark.parametrize("model,equilibrium", MODELS)
def test_initial_state_uses_the_model_equilibrium(lbm_lib, model, equilibrium):
    L, ref = make_pair(lbm_lib, 20, 20, 10, 8.0, precision="f64", omega=1.9, g=(0, 0, 2e-5),
                       model=model, equilibrium=equilibrium)
    L.init("loglaw", noise_amp=1e-3, seed=98)
    ref.init("loglaw", noise_amp=1e-3, seed=98)
    assert rel_err(L.populations(), ref.f) < 1e-14
    rho = 1.0 + 0.01 * np.random.default_rng(5).standard_normal((10, 20, 20))
    u = 0.02 * np.random.default_rng(6).standard_normal((3, 10, 20, 20))
    lbm_lib.lbm_init_fields(L.ctx, rho, u)
    ref.init_fields(rho, u)
    assert rel_err(L.populations(), ref.f, ref.fluid) < 1e-14
    L.close()


@pytest.mark.parametrize("model,equilibrium", MODELS)
def test_fp32_laminar_velocity_error(lbm_lib, model, equilibrium):
    """FP32 shifted storage: the same 1e-5 bound on the velocity after 1000 laminar steps
    as for the default model."""
    L, ref = make_pair(lbm_lib, 20, 20, 16, 8.0, precision="f32", wall="halfway", omega=1.25, g=(0, 0, 1e-5),
                       model=model, equilibrium=equilibrium)
    assert L.info()["variant"] == 2
    L.init("rest")
    ref.init("rest")
    L.step(1000)
    ref.step(1000)
    _, u = L.moments()
    _, uo = ref.moments()
    m = ref.fluid
    d = u.double().cpu().numpy()[:, m] - uo[:, m]
    assert float(np.sqrt(np.sum(d * d) / np.sum(uo[:, m] ** 2))) <= 1e-5
    L.close()


def test_statistics_and_graph_path(lbm_lib):
    """The statistics variant of the ablation kernel, and graph replays bit-identical to
    direct launches."""
    L, ref = make_pair(lbm_lib, 18, 18, 8, 7.0, precision="f64", omega=1.4, g=(0, 0, 1e-4),
                       model="bgk", equilibrium="order2")
    f0 = perturbed_state(ref, 414)
    L.set_populations(f0)
    lbm_lib.lbm_stats_enable(L.ctx, 3)
    ref.enable_stats(3)
    L.step(11)
    ref.step(11)
    acc = np.empty((4, 8, 18, 18))
    assert lbm_lib.lbm_stats_get(L.ctx, acc) == ref.stats_count == 4
    for k in range(4):
        assert np.max(np.abs(acc[k] - ref.stats[k])) < 1e-12 * np.max(np.abs(ref.stats[k]))
    L.close()

    A, _ = make_pair(lbm_lib, 18, 18, 8, 7.0, precision="f32", omega=1.4, g=(0, 0, 1e-4), model="bgk")
    B, _ = make_pair(lbm_lib, 18, 18, 8, 7.0, precision="f32", omega=1.4, g=(0, 0, 1e-4), model="bgk")
    for X in (A, B):
        X.init("laminar", noise_amp=1e-3, seed=3)
    lbm_lib.lbm_set_graph(B.ctx, 8)
    A.step(40)
    B.step(40)
    assert np.array_equal(A.populations(), B.populations())
    A.close()
    B.close()


def test_switching_models_and_errors(lbm_lib):
    lbm = lbm_lib
    L, ref = make_pair(lbm, 16, 16, 6, 6.0, precision="f32", omega=1.3)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_collision(L.ctx, 2, 0)
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_collision(L.ctx, 0, 5)
    assert e.value.status == lbm.LBM_EINVAL
    lbm.lbm_set_variant(L.ctx, 0)
    lbm.lbm_set_collision(L.ctx, "bgk", "hermite6")
    assert L.info()["variant"] == 2                    # the shape of the ablation kernels
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_variant(L.ctx, 1)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_autotune(L.ctx, 4)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adjoint(L.ctx, 4, lbm.LBM_J_UBULK, 0, None)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    # back to the default model: every launch shape again, and the default results
    lbm.lbm_set_collision(L.ctx, "mrt", "hermite6")
    lbm.lbm_set_variant(L.ctx, 1)
    L.init("laminar", noise_amp=1e-3, seed=4)
    ref.init("laminar", noise_amp=1e-3, seed=4)
    L.step(6)
    ref.step(6)
    assert rel_err(L.populations(), ref.f, ref.fluid) < 1e-6
    L.close()
    H, _ = make_pair(lbm, 16, 16, 6, 6.0, precision="f16s", omega=1.3)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_collision(H.ctx, "bgk", "hermite6")
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    H.close()


# ---- a general diagonal relaxation matrix --------------------------------------------------

def _rates(seed, omega):
    r = np.random.default_rng(seed).uniform(0.8, 1.9, 27)
    r[:4] = 1.0
    r[4:9] = omega
    return r


@pytest.mark.parametrize("equilibrium", ["hermite6", "order2"])
@pytest.mark.parametrize("wall", ["halfway", "bouzidi"])
def test_general_rates_parity(lbm_lib, equilibrium, wall):
    rates = _rates(7, 1.7)
    L, ref = make_pair(lbm_lib, 23, 19, 7, 7.3, precision="f64", wall=wall, omega=1.7, g=(2e-5, -1e-5, 3e-5),
                       trigger=dict(h=1e-4, period=20.0, modes=TRIG_MODES, t_end=100),
                       equilibrium=equilibrium, rates=rates)
    f0 = perturbed_state(ref, 121)
    L.set_populations(f0)
    for n in (1, 2, 3):
        L.step(n)
        ref.step(n)
        assert rel_err(L.populations(), ref.f, ref.fluid) < 1e-13, n
    L.close()


def test_paper_rates_through_the_general_transform_match_the_closed_form(lbm_lib):
    """The 27 x 27 transforms with Lambda of Eq. (lambda) against the closed-form kernel."""
    lbm = lbm_lib
    omega = 1.55
    rates = np.ones(27)
    rates[4:9] = omega
    A, ref = make_pair(lbm, 20, 20, 9, 8.2, precision="f64", omega=omega, g=(0, 0, 3e-5))
    B, _ = make_pair(lbm, 20, 20, 9, 8.2, precision="f64", omega=omega, g=(0, 0, 3e-5), rates=rates)
    f0 = perturbed_state(ref, 131)
    A.set_populations(f0)
    B.set_populations(f0)
    A.step(7)
    B.step(7)
    assert rel_err(B.populations(), A.populations(), ref.fluid) < 1e-13
    A.close()
    B.close()


def test_rates_in_an_ensemble_and_relax_updates(lbm_lib):
    """Members with and without rates in one launch, each against the oracle; lbm_set_relax
    switches a member between the two."""
    lbm = lbm_lib
    from oracle import lbm as O
    rates = _rates(9, 1.4)
    grids = [lbm.make_grid(18, 18, 6, 7.0, precision="f64", wall="halfway"),
             lbm.make_grid(14, 14, 6, 5.5, precision="f64", wall="halfway")]
    relaxes = [lbm.make_relax(1.4, rates), lbm.make_relax(1.2)]
    forces = [lbm.make_force(g=(0, 0, 2e-5)), lbm.make_force(g=(0, 0, 1e-5))]
    E = lbm.Lattice(None, None, ensemble=(grids, relaxes, forces))
    refs = [O.Run(18, 18, 6, omega=1.4, R=7.0, g=(0, 0, 2e-5), rates=rates),
            O.Run(14, 14, 6, omega=1.2, R=5.5, g=(0, 0, 1e-5))]
    for k, ref in enumerate(refs):
        E.select(k)
        E.set_populations(perturbed_state(ref, 140 + k))
    E.step(5)
    for k, ref in enumerate(refs):
        ref.step(5)
        E.select(k)
        assert rel_err(E.populations(), ref.f, ref.fluid) < 1e-13, k
    # member 0 back to the paper's matrix: the context returns to the closed-form kernel
    E.select(0)
    lbm.lbm_set_relax(E.ctx, lbm.make_relax(1.4))
    refs[0].rates = None
    E.step(3)
    for k, ref in enumerate(refs):
        ref.step(3)
        E.select(k)
        assert rel_err(E.populations(), ref.f, ref.fluid) < 1e-13, k
    E.close()


def test_rates_errors(lbm_lib):
    lbm = lbm_lib
    grid = lbm.make_grid(12, 12, 4, 4.5, precision="f32")
    bad = np.ones(27)
    bad[12] = 2.5
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(grid, lbm.make_relax(1.2, bad))
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(lbm.make_grid(12, 12, 4, 4.5, precision="bf16"), lbm.make_relax(1.2, np.ones(27)))
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    L = lbm.Lattice(grid, lbm.make_relax(1.2, np.ones(27)))
    assert L.info()["variant"] == 2
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adjoint(L.ctx, 4, lbm.LBM_J_UBULK, 0, None)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_relax(L.ctx, lbm.make_relax(1.2, bad))
    assert e.value.status == lbm.LBM_EINVAL
    L.close()
