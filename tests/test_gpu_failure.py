"""Failure detection and checkpoint/resume on the GPU, with failures made on the host.

* A non-finite population planted in a host copy and uploaded makes the periodic check
  return LBM_EUNSTABLE (no trap, the context stays usable).
* A run driven far beyond the method's stability range (omega = 1.99 with a huge body
  force) is caught by the check as LBM_EUNSTABLE.
* lbm_save / lbm_load resume bit-identically, statistics included.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pipe(lbm, omega=1.3, g=1e-5, precision="f32"):
    grid = lbm.make_grid(18, 18, 10, 7.0, precision=precision, wall="halfway")
    return lbm.Lattice(grid, lbm.lbm_relax(omega), lbm.make_force(g=(0.0, 0.0, g)))


def test_non_finite_population_is_reported(lbm_lib):
    lbm = lbm_lib
    L = _pipe(lbm)
    L.init("laminar", noise_amp=1e-4, seed=2)
    lbm.lbm_set_check(L.ctx, 4, 1e-6)
    L.step(8)
    f = L.populations()
    f[5, 4, 9, 9] = np.nan                       # a fluid cell near the axis
    L.set_populations(f)
    with pytest.raises(lbm.LbmError) as ei:
        L.step(8)
    assert ei.value.status == lbm.LBM_EUNSTABLE
    assert "non-finite" in str(ei.value)
    # the context is still usable: re-initialise and step
    L.init("rest")
    L.step(8)
    assert lbm.lbm_reduce(L.ctx)[4] == 0
    L.close()


def test_blow_up_is_reported(lbm_lib):
    lbm = lbm_lib
    L = _pipe(lbm, omega=1.99, g=0.02)
    L.init("rest")
    lbm.lbm_set_check(L.ctx, 10, 1e-3)
    with pytest.raises(lbm.LbmError) as ei:
        L.step(2000)
    assert ei.value.status == lbm.LBM_EUNSTABLE
    L.close()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_checkpoint_resume_is_bit_identical(lbm_lib, tmp_path, precision):
    lbm = lbm_lib
    L = _pipe(lbm, precision=precision)
    L.init("laminar", noise_amp=1e-3, seed=3)
    lbm.lbm_stats_enable(L.ctx, 2)
    L.step(7)                                    # odd t: reversed AA layout
    path = str(tmp_path / "state.lbm")
    lbm.lbm_save(L.ctx, path)
    L.step(6)
    fa = L.populations()
    acc_a = np.empty((4, 10, 18, 18))
    ca = lbm.lbm_stats_get(L.ctx, acc_a)
    M = _pipe(lbm, precision=precision)
    lbm.lbm_load(M.ctx, path)
    assert M.info()["t"] == 7
    M.step(6)
    acc_b = np.empty_like(acc_a)
    cb = lbm.lbm_stats_get(M.ctx, acc_b)
    assert np.array_equal(M.populations(), fa)
    assert ca == cb and np.array_equal(acc_a, acc_b)
    other = lbm.Lattice(lbm.make_grid(20, 20, 10, 8.0, precision=precision), lbm.lbm_relax(1.3))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_load(other.ctx, path)
    for x in (L, M, other):
        x.close()
