"""Error of every storage precision against FP64 storage in a turbulent window.

The point statistics of Sec. III.B (the radial profiles of the mean, u_rms, S3 and S4 of
u_z, lbm_stats_profile) of one window of a turbulent pipe are computed from the same
starting state with F64, F32, F16S and BF16 population storage:

1. spin-up: the pipe (by default the paper's 300 x 300 x 600 pipe of Sec. II.B) runs
   `spin` steps in F32 storage from the log-law start with the trigger force of Eq.
   (TurbForce) active for its first 3 T_LET;
2. the logical populations of the final (even) step are copied, as float64 on the
   device, into one context per storage precision (same grid and walls, body force only:
   the trigger is off by then, so restarting the step counter at 0 changes nothing);
3. each context runs `window` steps with FP64 statistics every `stats_every` steps, and
   its profiles are compared with the F64 context's: for every quantity X the error is
   max over radial bins |X_p - X_F64| / max over bins |X_F64|.

FP64 storage stands in for the FP64 oracle here: the numpy oracle cannot run a turbulent
window of a 42 M-cell pipe, and the library's F64 path matches it to 1e-12 per 100 steps.

  python -m paper_2405_12082_gb300.precision_study --workload paper --spin 6 --window 20000
"""
import argparse
import json
import sys
import time

import numpy as np

PRECISIONS = ("f64", "f32", "f16s", "bf16")
QUANTITIES = ("mean", "u_rms", "S3", "S4")


def make_lattice(lbm, cfg, precision, wall="halfway", trigger=True):
    from . import workloads as Wk
    grid = lbm.make_grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"], precision=precision, wall=wall)
    trig = None
    if trigger:
        trig = Wk.trigger_dict(h=cfg["h"], R=cfg["R"], nz=cfg["nz"], period=cfg["period"],
                               modes=cfg["trigger_modes"], t_end=cfg["t_trigger"])
    return lbm.Lattice(grid, lbm.lbm_relax(cfg["omega"]), lbm.make_force(g=(0.0, 0.0, cfg["h"]), trigger=trig))


def copy_state(lbm, src, cfg, precision, wall="halfway"):
    """A new context of the given storage precision holding the logical populations of
    `src` (at t = 0, body force only)."""
    import torch
    f = torch.empty((27, cfg["nz"], cfg["ny"], cfg["nx"]), dtype=torch.float64, device="cuda")
    lbm.lbm_get_populations(src.ctx, f)
    dst = make_lattice(lbm, cfg, precision, wall, trigger=False)
    lbm.lbm_set_populations(dst.ctx, f)
    del f
    torch.cuda.empty_cache()
    return dst


def window_profile(lbm, L, steps, stats_every, nbins, dr):
    lbm.lbm_stats_enable(L.ctx, stats_every)
    L.step(steps)
    prof = lbm.lbm_stats_profile(L.ctx, nbins, dr)
    bad = lbm.lbm_reduce(L.ctx)[4]
    return prof, bad


def compare(profiles, ref="f64"):
    """Relative error of every quantity of every precision against `ref` (bins with cells)."""
    p0 = profiles[ref]
    sel = p0[:, 1] > 0
    out = {}
    for p, prof in profiles.items():
        out[p] = {}
        for k, q in enumerate(QUANTITIES):
            a, b = prof[sel, 2 + k], p0[sel, 2 + k]
            scale = float(np.max(np.abs(b)))
            out[p][q] = float(np.max(np.abs(a - b)) / scale) if scale > 0 else float("nan")
    return out


def run(lbm, cfg, spin_steps, window, stats_every=100, nbins=None, dr=2.0, precisions=PRECISIONS,
        wall="halfway", log=None, reference="f64", control=False):
    """Spin-up, copy and windows; returns the profiles, the comparison against `reference`
    and timings.  control: the reference storage also runs the window that follows its
    first one ("<reference>:next"); its difference from the first window is the sampling
    error of a window of this length (the floor of any comparison)."""
    import torch
    nbins = nbins or int(cfg["R"] / dr)
    t0 = time.time()
    S = make_lattice(lbm, cfg, "f32", wall)
    S.init("loglaw", noise_amp=cfg["noise"], seed=20240520)
    spin_steps += spin_steps % 2
    S.step(spin_steps)
    _, u = S.moments()
    nf = S.info()["n_fluid"]
    state = {"spin_steps": spin_steps, "U_b": float(u[2].sum().item()) / nf,
             "max_u_r": float(torch.sqrt(u[0] ** 2 + u[1] ** 2).max().item()), "spin_s": time.time() - t0}
    del u
    if log:
        log(state)
    profiles, timings, bad = {}, {}, {}
    for p in precisions:
        L = copy_state(lbm, S, cfg, p, wall)
        t1 = time.time()
        profiles[p], bad[p] = window_profile(lbm, L, window, stats_every, nbins, dr)
        torch.cuda.synchronize()
        timings[p] = time.time() - t1
        if control and p == reference:
            key = p + ":next"
            profiles[key], bad[key] = window_profile(lbm, L, window, stats_every, nbins, dr)
        L.close()
        if log:
            log({"precision": p, "window_s": timings[p], "nonfinite": bad[p]})
    S.close()
    return {"state": state, "profiles": profiles, "errors": compare(profiles, reference), "window_s": timings,
            "nonfinite": bad, "reference": reference}


def main(argv=None):
    from . import lbm
    from . import workloads as Wk
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="paper", choices=["paper", "c2", "c3"])
    ap.add_argument("--spin", type=float, default=6.0, help="spin-up length in T_LET")
    ap.add_argument("--window", type=int, default=20000, help="compared window in steps")
    ap.add_argument("--stats-every", type=int, default=100)
    ap.add_argument("--wall", default="halfway", choices=["halfway", "bouzidi"])
    ap.add_argument("--precisions", default=",".join(PRECISIONS))
    ap.add_argument("--reference", default="f64", choices=list(PRECISIONS))
    ap.add_argument("--control", action="store_true",
                    help="also run the reference over the following window (sampling-error floor)")
    ap.add_argument("--out", default="precision_study.npz")
    a = ap.parse_args(argv)
    cfg = dict({"paper": Wk.C_PAPER, "c2": Wk.C2, "c3": Wk.C3}[a.workload])
    spin = int(round(a.spin * cfg["R"] / cfg["u_star"]))
    precs = tuple(p for p in a.precisions.split(",") if p)
    res = run(lbm, cfg, spin, a.window, a.stats_every, wall=a.wall, precisions=precs, reference=a.reference,
              control=a.control, log=lambda d: print(json.dumps(d), file=sys.stderr, flush=True))
    np.savez(a.out, **{"profile_" + p.replace(":", "_"): v for p, v in res["profiles"].items()})
    summary = {"workload": cfg["name"], "wall": a.wall, "spin_T_LET": a.spin, "window_steps": a.window,
               "stats_every": a.stats_every, "state": res["state"], "reference": a.reference,
               "errors_vs_reference": res["errors"], "window_s": res["window_s"], "nonfinite": res["nonfinite"],
               "profile_reference": res["profiles"][a.reference].tolist()}
    print(json.dumps(summary))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
