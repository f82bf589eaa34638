"""Turbulent pipe run following the protocol of Sec. II.B and Sec. III.C on the GPU.

The pipe (the paper's own 300 x 300 x 600 grid, or the R = 48 / R = 96 pipes at
Re_tau = 181.3, see workloads.py) starts from the mean
profile of Sec. II.B plus 5 % noise, is driven by the body force and, for the first
t_trigger steps, by the four-mode trigger force; after `total` large-eddy turnover times
(T_LET = R / u*) it has gathered point statistics every 100 steps and the dominant
azimuthal mode of u_z at 16 cross-sections every `modes_every` steps during the last
`window` turnover times.  Every number is computed by the library (kernels and its host
analysis functions); this script only drives the calls and writes an .npz and a JSON
summary (eigenvalues for the Chapman-Kolmogorov comparison come from numpy).

  python -m paper_2405_12082_gb300.run_pipe --workload c2 --total 30 --window 10 --out run.npz
"""
import argparse
import json
import math
import sys
import time

import numpy as np


def main(argv=None):
    from . import lbm
    from . import workloads as Wk
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="paper", choices=["paper", "c2", "c3"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f16s", "bf16"])
    ap.add_argument("--total", type=float, default=30.0, help="run length in T_LET")
    ap.add_argument("--steps", type=int, default=0, help="run length in steps (overrides --total)")
    ap.add_argument("--window", type=float, default=10.0, help="statistics window in T_LET (at the end)")
    ap.add_argument("--modes-every", type=int, default=20)
    ap.add_argument("--stats-every", type=int, default=100)
    ap.add_argument("--check-every", type=int, default=1000)
    ap.add_argument("--max-drift", type=float, default=1e-3,
                    help="stop when the mean density has moved by more than this")
    ap.add_argument("--wall", default="halfway", choices=["halfway", "bouzidi", "fullway"])
    ap.add_argument("--out", default="run.npz")
    a = ap.parse_args(argv)

    cfg = dict({"paper": Wk.C_PAPER, "c2": Wk.C2, "c3": Wk.C3}[a.workload])
    R, us, nu = cfg["R"], cfg["u_star"], cfg["nu"]
    t_let = R / us
    total = a.steps if a.steps > 0 else int(round(a.total * t_let))
    start = max(0, total - int(round(a.window * t_let)))
    start -= start % a.stats_every
    grid = lbm.make_grid(cfg["nx"], cfg["ny"], cfg["nz"], R, precision=a.precision, wall=a.wall)
    trig = Wk.trigger_dict(h=cfg["h"], R=R, nz=cfg["nz"], period=cfg["period"], modes=cfg["trigger_modes"],
                           t_end=cfg["t_trigger"])
    L = lbm.Lattice(grid, lbm.lbm_relax(cfg["omega"]), lbm.make_force(g=(0.0, 0.0, cfg["h"]), trigger=trig))
    L.init("loglaw", noise_amp=cfg["noise"], seed=Wk.SEED)
    lbm.lbm_set_check(L.ctx, a.check_every, a.max_drift)
    mass0 = lbm.lbm_reduce(L.ctx)[0]
    mcfg = lbm.make_modes_cfg(cfg["n_sections"], cfg["r_over_R"], cfg["n_theta"], cfg["n_modes"])
    n_samples = (total - start) // a.modes_every
    E = torch.empty((n_samples, cfg["n_sections"], 1, cfg["n_modes"] + 1), dtype=torch.float64, device="cuda")
    t0 = time.time()
    nf = L.info()["n_fluid"]
    chunk = max(a.modes_every, int(t_let) // 4)
    while L.info()["t"] < start:                       # progress: U_b / u* four times per T_LET
        L.step(min(chunk, start - L.info()["t"]))
        _, u = L.moments()
        print(json.dumps({"t": L.info()["t"], "U_b/u*": float(u[2].sum().item()) / nf / us,
                          "max|u_r|": float(torch.sqrt(u[0] ** 2 + u[1] ** 2).max().item())}),
              file=sys.stderr, flush=True)
    lbm.lbm_stats_enable(L.ctx, a.stats_every)
    ub = []
    for k in range(n_samples):
        lbm.lbm_modes(L.ctx, mcfg, E[k])
        L.step(a.modes_every)
        if k % max(1, n_samples // 50) == 0:
            _, u = L.moments()
            ub.append(float(u[2].sum().item()) / L.info()["n_fluid"])
    torch.cuda.synchronize()
    wall = time.time() - t0
    E_h = E.cpu().numpy()
    kstar = np.stack([lbm.lbm_dominant_modes(E_h[k], 0, 1, 10) for k in range(n_samples)])   # [time][section]
    # every cross-section gives its own series; counts and correlations are pooled
    ns = kstar.shape[1]
    counts = sum(lbm.lbm_transition_matrix(kstar[:, s], 1, 10, 1)[1] for s in range(ns))
    T1 = counts / np.maximum(counts.sum(axis=0, keepdims=True), 1)
    ck = {}
    for d in range(1, 6):
        cd = sum(lbm.lbm_transition_matrix(kstar[:, s], 1, 10, d)[1] for s in range(ns))
        Td = cd / np.maximum(cd.sum(axis=0, keepdims=True), 1)
        ck[d] = {"decimated": sorted(np.abs(np.linalg.eigvals(Td)).tolist(), reverse=True),
                 "power": sorted(np.abs(np.linalg.eigvals(np.linalg.matrix_power(T1, d))).tolist(), reverse=True)}
    max_lag = min(300, n_samples - 1)
    F = sum(lbm.lbm_mode_correlation(kstar[:, s], 1, 10, max_lag) for s in range(ns)) / ns
    prof = lbm.lbm_stats_profile(L.ctx, int(R / 2), 2.0)
    delta_plus = (R - prof[:, 0]) * us / nu
    Ub = float(np.mean(ub[len(ub) // 2:])) if ub else float("nan")
    hist = np.bincount(kstar.ravel(), minlength=11)[1:11]
    summary = {
        "workload": cfg["name"], "precision": a.precision, "wall": a.wall, "steps": total, "stats_from": start,
        "mean_density_change": (lbm.lbm_reduce(L.ctx)[0] - mass0) / nf,
        "T_LET": t_let, "Re_tau": us * R / nu, "wall_s": wall,
        "U_b": Ub, "U_b_over_u_star": Ub / us, "Re_bulk": Ub * 2 * R / nu,
        "mode_pdf": (hist / max(hist.sum(), 1)).tolist(),
        "transition_diag": np.diag(T1).tolist(),
        "ck_eigs": ck, "F_mean_over_modes": F.mean(axis=0)[:: max(1, max_lag // 30)].tolist(),
        "profile_u_plus_at_delta_plus": [
            [float(dp), float(m / us), float(r / us), float(s3), float(s4)]
            for dp, m, r, s3, s4 in zip(delta_plus, prof[:, 2], prof[:, 3], prof[:, 4], prof[:, 5])
            if prof[0, 1] >= 0],
    }
    np.savez(a.out, kstar=kstar, T1=T1, counts=counts, F=F, profile=prof, delta_plus=delta_plus,
             ub=np.array(ub), E_last=E_h[-1])
    L.close()
    print(json.dumps(summary))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
