"""Oracle recomputation of single cells of a full-size state (test infrastructure).

The numpy oracle cannot step a pipe of millions of cells, but one step of a few hundred
cells needs only their 27 upstream neighbours: collide each source cell with the literal
moment-space collision (oracle.collision.collide) and stream by pull with half-way walls.
`fetch(z, y, x)` returns the previous populations of the given cells as [27, n] float64.
"""
import numpy as np

from oracle import lbm as O
from oracle.collision import collide, macroscopic
from oracle.lattice import C, OPP


def accel(cfg, tr, z, y, x, t):
    """Acceleration g(x, t) of the workload (constant h plus the trigger force)."""
    xc, yc = (cfg["nx"] - 1) / 2.0, (cfg["ny"] - 1) / 2.0
    fx, fy, fz = tr.cartesian(x - xc, y - yc, np.asarray(z).astype(float), t)
    return np.array([fx, fy, fz + cfg["h"]])


def oracle_trigger(cfg):
    return O.Trigger(h=cfg["h"], R=cfg["R"], L=cfg["nz"], period=cfg["period"], modes=cfg["trigger_modes"],
                     t_end=cfg["t_trigger"])


def one_step(cfg, tr, fetch, t, fluid, z, y, x):
    """f(t+1) at the cells (z, y, x) from the state f(t): pull from x - c_i, half-way walls."""
    nz, ny, nx = fluid.shape
    srcs = []
    for i in range(27):
        cx, cy, cz = (int(v) for v in C[i])
        zs, ys, xs = (z - cz) % nz, (y - cy) % ny, (x - cx) % nx
        src_fluid = fluid[zs, ys, xs]
        srcs.append((np.where(src_fluid, zs, z), np.where(src_fluid, ys, y), np.where(src_fluid, xs, x), src_fluid))
    allz = np.concatenate([s[0] for s in srcs])
    ally = np.concatenate([s[1] for s in srcs])
    allx = np.concatenate([s[2] for s in srcs])
    g = accel(cfg, tr, allz, ally, allx, t)
    fs = collide(fetch(allz, ally, allx), g, cfg["omega"])
    n = len(x)
    out = np.empty((27, n))
    for i in range(27):
        block = fs[:, i * n:(i + 1) * n]
        out[i] = np.where(srcs[i][3], block[i], block[OPP[i]])
    return out


def uz_before_collision(cfg, tr, fetch, t, z, y, x):
    """u_z of Eq. (macroscopic_u) with the force of step t, from f(t) at the given cells."""
    g = accel(cfg, tr, z, y, x, t)
    _, u = macroscopic(fetch(z, y, x), g)
    return u[2]


def device_fetch(fdev):
    """fetch() over a torch tensor [27, nz, ny, nx] of float64 on the device."""
    import torch

    def f(z, y, x):
        idx = [torch.as_tensor(np.asarray(a, dtype=np.int64), device=fdev.device) for a in (z, y, x)]
        return fdev[:, idx[0], idx[1], idx[2]].cpu().numpy()
    return f


def host_fetch(f):
    return lambda z, y, x: f[:, z, y, x]
