"""Helpers that set up the same seeded problem on the CUDA library and on the oracle."""
import numpy as np

from oracle import lbm as O
from paper_2405_12082_gb300 import workloads as Wk

TRIG_MODES = [(1, 0.3, 0.4), (2, 0.4, 0.0), (3, 0.3, 1.3)]


def oracle_trigger(h, R, nz, period, modes, t_end):
    return O.Trigger(h=h, R=R, L=nz, A0=50.0, kappa=0.5, kz=3, period=period, l0=0.2 * R, l=0.4 * R,
                     modes=modes, t_end=t_end)


def make_pair(lbm, nx, ny, nz, R, precision="f64", wall="halfway", omega=1.3, g=(0.0, 0.0, 1e-5),
              trigger=None, gz=None, geometry="pipe", f16_log2_scale=0, model="mrt", equilibrium="hermite6",
              rates=None):
    """trigger: None or dict(h, period, modes, t_end); gz: None or a float64 (nz, ny, nx) field;
    model / equilibrium / rates: the collision model of both sides."""
    grid = lbm.make_grid(nx, ny, nz, R, geometry=geometry, precision=precision, wall=wall,
                         f16_log2_scale=f16_log2_scale)
    tr_dev = tr_or = None
    if trigger is not None:
        tr_dev = Wk.trigger_dict(h=trigger["h"], R=R, nz=nz, period=trigger["period"], modes=trigger["modes"],
                                 t_end=trigger["t_end"])
        tr_or = oracle_trigger(trigger["h"], R, nz, trigger["period"], trigger["modes"], trigger["t_end"])
    gz_dev = None
    if gz is not None:
        import torch
        dt = torch.float64 if precision == "f64" else torch.float32
        gz_dev = torch.tensor(gz, dtype=dt, device="cuda").contiguous()
        if precision != "f64":
            gz = gz_dev.double().cpu().numpy()      # the oracle sees exactly the stored values
    force = lbm.make_force(g=g, trigger=tr_dev, gz_field=gz_dev)
    L = lbm.Lattice(grid, lbm.make_relax(omega, rates), force)
    L._keep.append(gz_dev)
    if (model, equilibrium) != ("mrt", "hermite6"):
        lbm.lbm_set_collision(L.ctx, model, equilibrium)
    ref = O.Run(nx, ny, nz, omega=omega, R=R if geometry == "pipe" else None, geometry=geometry, wall=wall,
                g=g, trigger=tr_or, gz_field=gz, model=model, equilibrium=equilibrium, rates=rates)
    return L, ref


def perturbed_state(ref, seed, u_amp=0.03, rho_amp=0.01, f_amp=1e-3):
    """A seeded non-equilibrium state: f^eq(rho, u) of random fields plus noise (fluid cells)."""
    shp = (ref.nz, ref.ny, ref.nx)
    rho = 1.0 + Wk.perturbation(shp, seed, rho_amp)
    u = Wk.random_velocity(shp, seed + 1, u_amp)
    ref.init_fields(rho, u)
    f = ref.f + Wk.perturbation(ref.f.shape, seed + 2, f_amp) * (ref.fluid[None] if ref.geometry == "pipe" else 1)
    ref.f = f.copy()
    return f


def rel_err(a, b, mask=None):
    if mask is not None:
        a = a[:, mask]
        b = b[:, mask]
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
