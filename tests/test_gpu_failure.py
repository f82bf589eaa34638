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


# byte offsets in the checkpoint header: magic[8], then int32 precision, wall, n_members,
# stats_every, then int64 stride, dense_total, t, stats_count, pop_bytes, stats_bytes
_HDR = {"stats_every": (20, "<i4"), "t": (40, "<i8"), "stats_count": (48, "<i8"), "stats_bytes": (64, "<i8")}


def _doctor(src, dst, field, value):
    data = bytearray(open(src, "rb").read())
    off, fmt = _HDR[field]
    data[off:off + np.dtype(fmt).itemsize] = np.array([value], dtype=fmt).tobytes()
    open(dst, "wb").write(bytes(data))


@pytest.mark.parametrize("field,value", [("stats_bytes", 1 << 40), ("stats_bytes", -8), ("stats_bytes", 8),
                                         ("stats_every", 0), ("stats_count", -1), ("t", -2)])
def test_load_rejects_a_doctored_header(lbm_lib, tmp_path, field, value):
    """A checkpoint whose header was altered on the host is rejected with LBM_EINVAL before
    any byte reaches the device: the context keeps its populations, t and statistics."""
    lbm = lbm_lib
    L = _pipe(lbm)
    L.init("laminar", noise_amp=1e-3, seed=4)
    lbm.lbm_stats_enable(L.ctx, 2)
    L.step(5)
    good = str(tmp_path / "good.lbm")
    lbm.lbm_save(L.ctx, good)
    M = _pipe(lbm)
    M.init("laminar", noise_amp=1e-3, seed=8)
    lbm.lbm_stats_enable(M.ctx, 3)
    M.step(4)
    before = M.populations()
    acc0 = np.empty((4, 10, 18, 18))
    c0 = lbm.lbm_stats_get(M.ctx, acc0)
    bad = str(tmp_path / "bad.lbm")
    _doctor(good, bad, field, value)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_load(M.ctx, bad)
    assert ei.value.status == lbm.LBM_EINVAL
    assert M.info()["t"] == 4
    assert np.array_equal(M.populations(), before)
    acc1 = np.empty_like(acc0)
    assert lbm.lbm_stats_get(M.ctx, acc1) == c0 and np.array_equal(acc0, acc1)
    L.close()
    M.close()


def test_load_rejects_a_truncated_file(lbm_lib, tmp_path):
    lbm = lbm_lib
    L = _pipe(lbm)
    L.init("laminar", noise_amp=1e-3, seed=4)
    lbm.lbm_stats_enable(L.ctx, 2)
    L.step(3)
    good = str(tmp_path / "good.lbm")
    lbm.lbm_save(L.ctx, good)
    data = open(good, "rb").read()
    M = _pipe(lbm)
    M.init("rest")
    before = M.populations()
    for cut in (len(data) - 8, 72 + 100, 40):        # inside the statistics, the populations, the header
        bad = str(tmp_path / ("cut%d.lbm" % cut))
        open(bad, "wb").write(data[:cut])
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_load(M.ctx, bad)
        assert ei.value.status == lbm.LBM_EINVAL
        assert M.info()["t"] == 0
        assert np.array_equal(M.populations(), before)
    L.close()
    M.close()
