"""Adjoint step on the GPU: against the FP64 oracle adjoint and against finite differences.

* FP64 library adjoint = oracle adjoint (complex-step Jacobians of the literal step) for
  both objectives, with ragged checkpoint segments: J to 1e-12, gradients to 1e-10.
* FP32 adjoint of the 52 x 52 x 256, R = 24 pipe over 2000 steps (tau = 0.8, per-cell
  axial acceleration 1e-6) against central differences with h = 1e-4 of the FP64 forward,
  on 32 seeded cells and on omega: relative agreement 1e-4.
* After lbm_adjoint the context holds exactly the state of a plain forward run.
"""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import lbm as O
from paper_2405_12082_gb300 import workloads as Wk

pytestmark = pytest.mark.gpu


def _ctx(lbm, nx, nz, R, omega, g, gz, precision):
    import torch
    dt = torch.float64 if precision == "f64" else torch.float32
    gzd = torch.tensor(gz, dtype=dt, device="cuda").contiguous()
    grid = lbm.make_grid(nx, nx, nz, R, precision=precision, wall="halfway")
    L = lbm.Lattice(grid, lbm.lbm_relax(omega), lbm.make_force(g=g, gz_field=gzd))
    L._keep.append(gzd)
    return L


@pytest.mark.parametrize("objective,every", [("ubulk", 3), ("wss", 3), ("ubulk", 10), ("wss", 0)])
def test_fp64_adjoint_matches_the_oracle(lbm_lib, objective, every):
    """every = 3: four segments, the last of one step; 10: a single segment (all moments
    stored by the forward pass); 0: ceil(sqrt(10)) = 4, segments of 4, 4, 2."""
    lbm = lbm_lib
    nx, nz, R, omega, T = 14, 6, 5.5, 1.3, 10
    g = (0.0, 0.0, 1e-5)
    gz = Wk.gz_field(nz, nx, nx, base=1e-4, seed=77, rel_amp=0.5)
    run = O.Run(nx, nx, nz, omega=omega, R=R, wall="halfway", g=g, gz_field=gz)
    run.init_fields(np.ones((nz, nx, nx)), Wk.random_velocity((nz, nx, nx), 78, 0.01))
    run.f = run.f + Wk.perturbation(run.f.shape, 79, 1e-4) * run.fluid[None]
    f0 = run.f.copy()
    L = _ctx(lbm, nx, nz, R, omega, g, gz, "f64")
    L.set_populations(f0)
    dgz = np.zeros((nz, nx, nx))
    obj = lbm.LBM_J_UBULK if objective == "ubulk" else lbm.LBM_J_WSS
    J, dw = lbm.lbm_adjoint(L.ctx, T, obj, every, dgz)
    Jo, dgzo, dwo = A.adjoint(run, T, objective)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    m = run.fluid
    assert np.max(np.abs(dgz[m] - dgzo[m])) <= 1e-10 * np.max(np.abs(dgzo[m]))
    assert np.all(dgz[~m] == 0)
    assert abs(dw - dwo) <= 1e-10 * abs(dwo)
    # the context now holds the state after T steps
    assert np.max(np.abs(L.populations()[:, m] - run.f[:, m])) <= 1e-13
    assert L.info()["t"] == T
    L.close()


def _J_forward_ubulk(lbm, c, gz, omega, T, f64_ctx_cache):
    """J of the bulk-velocity objective from an FP64 forward run: the FP64 sums of u_z at
    every step t = 0..T-1 (statistics sampled every step) averaged over cells and steps."""
    L = _ctx(lbm, c["nx"], c["nz"], c["R"], omega, (0.0, 0.0, 0.0), gz, "f64")
    L.init("rest")
    lbm.lbm_stats_enable(L.ctx, 1)
    L.step(T)
    acc = np.empty((4, c["nz"], c["ny"], c["nx"]))
    count = lbm.lbm_stats_get(L.ctx, acc)
    n_fluid = L.info()["n_fluid"]
    L.close()
    assert count == T
    return acc[0].sum() / (T * n_fluid)


def test_fp32_adjoint_matches_central_differences_on_the_adjoint_pipe(lbm_lib):
    lbm = lbm_lib
    c = Wk.C5
    T, h = c["T"], 1e-4
    gz = np.full((c["nz"], c["ny"], c["nx"]), c["gz"])
    L = _ctx(lbm, c["nx"], c["nz"], c["R"], c["omega"], (0.0, 0.0, 0.0), gz, "f32")
    L.init("rest")
    dgz = np.zeros_like(gz)
    J, dw = lbm.lbm_adjoint(L.ctx, T, lbm.LBM_J_UBULK, 0, dgz)
    mask = np.zeros(gz.shape, dtype=bool)
    fm = np.empty((c["ny"], c["nx"]), dtype=np.uint8)
    lbm.lbm_fluid_mask(L.ctx, fm)
    mask[:] = fm.astype(bool)[None]
    L.close()
    J64 = _J_forward_ubulk(lbm, c, gz, c["omega"], T, None)
    assert abs(J - J64) <= 1e-5 * abs(J64)
    cells = Wk.choose_cells(mask, 32, seed=Wk.SEED)
    for cell in cells:
        idx = np.unravel_index(cell, gz.shape)
        gp, gm = gz.copy(), gz.copy()
        gp[idx] += h
        gm[idx] -= h
        fd = (_J_forward_ubulk(lbm, c, gp, c["omega"], T, None) - _J_forward_ubulk(lbm, c, gm, c["omega"], T, None)) / (2 * h)
        assert abs(dgz[idx] - fd) <= 1e-4 * abs(fd), (cell, dgz[idx], fd)
    fd = (_J_forward_ubulk(lbm, c, gz, c["omega"] + h, T, None) - _J_forward_ubulk(lbm, c, gz, c["omega"] - h, T, None)) / (2 * h)
    assert abs(dw - fd) <= 1e-4 * abs(fd), (dw, fd)


def test_fp32_wall_shear_adjoint_against_fp64(lbm_lib):
    """The wall-shear gradient of the FP32 sweep against the FP64 sweep (itself matched to the
    oracle above) on a shorter run of the adjoint pipe's cross-section."""
    lbm = lbm_lib
    c = Wk.C5
    nz, T = 32, 400
    gz = Wk.gz_field(nz, c["ny"], c["nx"], base=c["gz"], seed=5, rel_amp=0.3)
    out = {}
    for prec in ("f32", "f64"):
        L = _ctx(lbm, c["nx"], nz, c["R"], c["omega"], (0.0, 0.0, 0.0), gz, prec)
        L.init("rest")
        d = np.zeros_like(gz)
        J, dw = lbm.lbm_adjoint(L.ctx, T, lbm.LBM_J_WSS, 20, d)
        out[prec] = (J, d, dw)
        L.close()
    J32, d32, w32 = out["f32"]
    J64, d64, w64 = out["f64"]
    assert abs(J32 - J64) <= 1e-4 * abs(J64)
    assert np.max(np.abs(d32 - d64)) <= 1e-4 * np.max(np.abs(d64))
    assert abs(w32 - w64) <= 1e-4 * abs(w64)


def test_adjoint_leaves_the_forward_state(lbm_lib):
    lbm = lbm_lib
    gz = Wk.gz_field(8, 20, 20, base=2e-5, seed=3, rel_amp=0.2)
    states = []
    for run_adjoint in (False, True):
        L = _ctx(lbm, 20, 8, 8.0, 1.4, (0.0, 0.0, 1e-5), gz, "f32")
        L.init("laminar", noise_amp=1e-3, seed=8)
        if run_adjoint:
            lbm.lbm_adjoint(L.ctx, 25, lbm.LBM_J_UBULK, 4, np.zeros_like(gz))
        else:
            L.step(25)
        states.append((L.populations(), L.info()["t"]))
        L.close()
    assert states[0][1] == states[1][1] == 25
    assert np.array_equal(states[0][0], states[1][0])


def test_adjoint_rejects_a_trigger(lbm_lib):
    lbm = lbm_lib
    grid = lbm.make_grid(16, 16, 8, 6.0, precision="f32", wall="halfway")
    trig = Wk.trigger_dict(h=1e-5, R=6.0, nz=8, period=50.0, modes=[(2, 1.0, 0.0)], t_end=100)
    L = lbm.Lattice(grid, lbm.lbm_relax(1.3), lbm.make_force(g=(0, 0, 1e-5), trigger=trig))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adjoint(L.ctx, 4, lbm.LBM_J_UBULK, 0, None)
    assert e.value.status == lbm.LBM_EUNSUPPORTED
    L.close()


def test_autograd_wrapper_returns_the_adjoint_gradients(lbm_lib):
    """pipe_objective(...).backward() hands back exactly what lbm_adjoint computes."""
    import torch
    lbm = lbm_lib
    nx, nz, R, T = 16, 8, 6.5, 30
    gz0 = Wk.gz_field(nz, nx, nx, base=2e-5, seed=12, rel_amp=0.3)
    runs = []
    for mode in ("direct", "autograd"):
        L = _ctx(lbm, nx, nz, R, 1.3, (0.0, 0.0, 0.0), gz0, "f64")
        L.init("laminar", noise_amp=1e-4, seed=13)
        if mode == "direct":
            d = np.zeros((nz, nx, nx))
            J, dw = lbm.lbm_adjoint(L.ctx, T, lbm.LBM_J_UBULK, 0, d)
            runs.append((J, d, dw))
        else:
            gz = torch.tensor(gz0, dtype=torch.float64, device="cuda", requires_grad=True)
            om = torch.tensor(1.3, dtype=torch.float64, requires_grad=True)
            Jt = lbm.pipe_objective(L, gz, om, T, "ubulk")
            Jt.backward()
            runs.append((float(Jt.item()), gz.grad.cpu().numpy(), float(om.grad.item())))
        L.close()
    (J0, d0, w0), (J1, d1, w1) = runs
    assert J0 == J1
    assert np.array_equal(d0, d1)
    assert w0 == w1
