"""Element-wise parity of the compressed storages and of the FP32 statistics path at the
full workload sizes, in the launch shape each storage runs by default (the one bench.py
times), and a finite-difference check of the wall-shear adjoint on the adjoint pipe.

* F16S and BF16 storage on the R = 48 (100 x 100 x 480) and R = 96 (196 x 196 x 1152)
  pipes with the four-mode trigger: one even and one odd step of 400 sampled cells,
  recomputed by the FP64 oracle from the GPU's own decoded previous state.  The GPU
  collides in FP32 and rounds f - w to the storage format once per store, so each
  population may differ by one rounding of the format, 2^-11 |f - w| (half, 11-bit
  significand; the 2^16 scale is exact) or 2^-8 |f - w| (bfloat16), plus twice the FP32
  collision error bound used for F32 storage (2e-8).
* F32 storage with statistics on every step: the FP64 sums of u_z^k, k = 1..4, after an
  even and an odd sample step, on 400 sampled cells, against u_z of the oracle from the
  GPU's own decoded states (FP32 rounding of u_z, at most 2e-7 here, propagated to u^k).
* Wall-shear objective of the adjoint pipe (52 x 52 x 256, T = 2000, FP32 adjoint)
  against central differences (h = 1e-4) of the FP64 objective on 6 seeded cells and on
  omega: 1e-4 relative.
"""
import numpy as np
import pytest

from oracle import lbm as O
from oracle.lattice import W
from paper_2405_12082_gb300 import workloads as Wk

import _sampled as S

pytestmark = pytest.mark.gpu

STORAGE_ROUNDING = {"f16s": 2.0 ** -11, "bf16": 2.0 ** -8}
F32_COLLISION = 2e-8


def _pipe(lbm, cfg, precision, stats_every=0):
    grid = lbm.make_grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"], precision=precision, wall="halfway")
    trig = Wk.trigger_dict(h=cfg["h"], R=cfg["R"], nz=cfg["nz"], period=cfg["period"], modes=cfg["trigger_modes"],
                           t_end=cfg["t_trigger"])
    L = lbm.Lattice(grid, lbm.lbm_relax(cfg["omega"]), lbm.make_force(g=(0.0, 0.0, cfg["h"]), trigger=trig))
    L.init("loglaw", noise_amp=cfg["noise"], seed=Wk.SEED)
    if stats_every:
        lbm.lbm_stats_enable(L.ctx, stats_every)
    return L


def _device_populations(lbm, L, cfg):
    import torch
    f = torch.empty((27, cfg["nz"], cfg["ny"], cfg["nx"]), dtype=torch.float64, device="cuda")
    lbm.lbm_get_populations(L.ctx, f)
    return f


@pytest.mark.parametrize("wl", ["c2", "c3"])
@pytest.mark.parametrize("precision", ["f16s", "bf16"])
def test_compressed_storage_one_step_on_sampled_cells(lbm_lib, wl, precision):
    import torch
    lbm = lbm_lib
    cfg = {"c2": Wk.C2, "c3": Wk.C3}[wl]
    L = _pipe(lbm, cfg, precision)
    info = L.info()
    states = [_device_populations(lbm, L, cfg)]
    for _ in range(2):
        L.step(1)
        states.append(_device_populations(lbm, L, cfg))
    assert lbm.lbm_reduce(L.ctx)[4] == 0
    L.close()
    fluid = O.fluid_mask(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"])
    tr = S.oracle_trigger(cfg)
    eps = STORAGE_ROUNDING[precision]
    for step in (0, 1):                        # even (t = 0 -> 1) and odd (t = 1 -> 2) AA steps
        cells = Wk.choose_cells(fluid, 400, 10 + step)
        z, y, x = np.unravel_index(cells, fluid.shape)
        expect = S.one_step(cfg, tr, S.device_fetch(states[step]), step, fluid, z, y, x)
        got = S.device_fetch(states[step + 1])(z, y, x)
        shifted = np.abs(expect - W[:, None])
        bound = eps * shifted + 2 * F32_COLLISION
        err = np.abs(got - expect)
        assert np.all(err <= bound), (wl, precision, step, info["variant"], float(np.max(err / bound)))
        # the rounding is really that of the format (not far below it): the stored values
        # are not FP32 in disguise
        assert np.max(err) > 0.05 * eps * np.max(shifted)
    del states
    torch.cuda.empty_cache()


def test_fp32_statistics_path_on_sampled_cells(lbm_lib):
    """Statistics every step from t = 0: after two steps the sums hold u_z^k of t = 0
    (even step kernel with statistics) and of t = 1 (odd step kernel with statistics)."""
    import torch
    lbm = lbm_lib
    cfg = Wk.C2
    L = _pipe(lbm, cfg, "f32", stats_every=1)
    f0 = _device_populations(lbm, L, cfg)
    L.step(1)
    f1 = _device_populations(lbm, L, cfg)
    L.step(1)
    acc = torch.empty((4, cfg["nz"], cfg["ny"], cfg["nx"]), dtype=torch.float64, device="cuda")
    count = lbm.lbm_stats_get(L.ctx, acc)
    L.close()
    assert count == 2
    fluid = O.fluid_mask(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"])
    tr = S.oracle_trigger(cfg)
    cells = Wk.choose_cells(fluid, 400, 21)
    z, y, x = np.unravel_index(cells, fluid.shape)
    u0 = S.uz_before_collision(cfg, tr, S.device_fetch(f0), 0, z, y, x)
    u1 = S.uz_before_collision(cfg, tr, S.device_fetch(f1), 1, z, y, x)
    got = S.device_fetch(acc)(z, y, x)
    du = 2e-7
    for k in range(1, 5):
        expect = u0 ** k + u1 ** k
        bound = k * (np.abs(u0) ** (k - 1) + np.abs(u1) ** (k - 1)) * du * 1.01 + 1e-300
        assert np.all(np.abs(got[k - 1] - expect) <= bound), (k, float(np.max(np.abs(got[k - 1] - expect) / bound)))
    # solid cells never accumulate
    solid = ~fluid
    assert float(acc[:, torch.as_tensor(solid, device="cuda")].abs().max().item()) == 0.0


def _adj_ctx(lbm, c, gz, omega, precision):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    gzd = torch.tensor(gz, dtype=dt, device="cuda").contiguous()
    grid = lbm.make_grid(c["nx"], c["ny"], c["nz"], c["R"], precision=precision, wall="halfway")
    L = lbm.Lattice(grid, lbm.lbm_relax(omega), lbm.make_force(gz_field=gzd))
    L._keep.append(gzd)
    return L


def _J_wss_f64(lbm, c, gz, omega, T):
    """The FP64 wall-shear objective of a forward run from rest: J of an FP64 lbm_adjoint call
    (the FP64 J equals the oracle's J to 1e-12, test_gpu_adjoint.py)."""
    L = _adj_ctx(lbm, c, gz, omega, "f64")
    L.init("rest")
    J, _ = lbm.lbm_adjoint(L.ctx, T, lbm.LBM_J_WSS, 0, None)
    L.close()
    return J


def test_fp32_wall_shear_adjoint_matches_central_differences(lbm_lib):
    lbm = lbm_lib
    c = Wk.C5
    T, h = c["T"], 1e-4
    gz = np.full((c["nz"], c["ny"], c["nx"]), c["gz"])
    L = _adj_ctx(lbm, c, gz, c["omega"], "f32")
    L.init("rest")
    dgz = np.zeros_like(gz)
    J, dw = lbm.lbm_adjoint(L.ctx, T, lbm.LBM_J_WSS, 0, dgz)
    fm = np.empty((c["ny"], c["nx"]), dtype=np.uint8)
    lbm.lbm_fluid_mask(L.ctx, fm)
    L.close()
    mask = np.broadcast_to(fm.astype(bool)[None], gz.shape)
    J64 = _J_wss_f64(lbm, c, gz, c["omega"], T)
    assert abs(J - J64) <= 1e-5 * abs(J64)
    for cell in Wk.choose_cells(mask, 6, seed=Wk.SEED + 5):
        idx = np.unravel_index(cell, gz.shape)
        gp, gm = gz.copy(), gz.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (_J_wss_f64(lbm, c, gp, c["omega"], T) - _J_wss_f64(lbm, c, gm, c["omega"], T)) / (2 * h)
        assert abs(dgz[idx] - fd) <= 1e-4 * abs(fd), (cell, dgz[idx], fd)
    fd = (_J_wss_f64(lbm, c, gz, c["omega"] + h, T) - _J_wss_f64(lbm, c, gz, c["omega"] - h, T)) / (2 * h)
    assert abs(dw - fd) <= 1e-4 * abs(fd), (dw, fd)
