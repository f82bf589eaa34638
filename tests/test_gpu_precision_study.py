"""The machinery of the turbulent precision comparison (precision_study.py) on a small
pipe in a few hundred steps: the state copied into another storage is the source state
(exactly for F32 and F64, to the format's rounding for F16S and BF16), F64 compared with
itself has zero error, every window stays finite, and F32 storage differs from F64
storage by FP32 rounding only over this short, mildly perturbed window."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CFG = dict(name="small pipe 40x40x32 R=17", nx=40, ny=40, nz=32, R=17.0, omega=1.8, h=2e-5, period=60.0,
           t_trigger=150, noise=0.01, trigger_modes=[(2, 1.0, 0.0)], u_star=0.004)


def test_state_copy_between_storages(lbm_lib):
    from paper_2405_12082_gb300 import precision_study as PS
    lbm = lbm_lib
    S = PS.make_lattice(lbm, CFG, "f32")
    S.init("loglaw", noise_amp=CFG["noise"], seed=3)
    S.step(10)
    f = S.populations()
    fluid = np.zeros((CFG["nz"], CFG["ny"], CFG["nx"]), dtype=bool)
    m = np.empty((CFG["ny"], CFG["nx"]), dtype=np.uint8)
    lbm.lbm_fluid_mask(S.ctx, m)
    fluid[:] = m.astype(bool)[None]
    from oracle.lattice import W
    for p, rel in (("f64", 0.0), ("f32", 0.0), ("f16s", 2.0 ** -11), ("bf16", 2.0 ** -8)):
        L = PS.copy_state(lbm, S, CFG, p)
        assert L.info()["t"] == 0
        g = L.populations()
        d = np.abs(g[:, fluid] - f[:, fluid])
        # (+1e-12: the half format is subnormal below 2^-14, i.e. |f - w| < 2^-30 at the 2^16 scale)
        assert np.all(d <= rel * np.abs(f[:, fluid] - W[:, None]) + 1e-12), p
        L.close()
    S.close()


def test_window_comparison_runs_and_is_consistent(lbm_lib):
    from paper_2405_12082_gb300 import precision_study as PS
    res = PS.run(lbm_lib, CFG, spin_steps=200, window=300, stats_every=5, nbins=8, dr=2.0)
    assert set(res["errors"]) == set(PS.PRECISIONS)
    for q in PS.QUANTITIES:
        assert res["errors"]["f64"][q] == 0.0
        assert res["errors"]["f32"][q] < 1e-3, (q, res["errors"]["f32"])
        for p in PS.PRECISIONS:
            assert np.isfinite(res["errors"][p][q]), (p, q)
    assert all(v == 0 for v in res["nonfinite"].values())
    prof = res["profiles"]["f64"]
    assert np.all(prof[prof[:, 1] > 0, 3] > 0)        # fluctuations were sampled (u_rms > 0)
