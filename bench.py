"""Throughput of the fused D3Q27 MRT pipe step on one GB300 (JSON line on stdout).

Workload (default): the R = 48 turbulent pipe, 100 x 100 x 480 cells, FP32 shifted
populations, Re_tau = 181.3 parameters, log-law start with 5 % Gaussian noise, the
four-mode trigger force active, FP64 statistics every 100 steps and the 16-section
azimuthal mode analysis every 100 steps.  One bench step = 100 lattice steps (one of
them with the fused statistics accumulation) + one mode analysis, i.e. every row
of the hot path.  The population array (518 MB) is larger than L2, so no flush is
needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c2|c3] [--precision f32|f16s|bf16|f64]

Under torchrun (N > 1) every rank runs its own replica of the pipe on its own GPU
(the path has no exchange step); rank 0 prints the aggregate.
`--impl reference` times the FP64 oracle on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2405_12082_gb300 import workloads as Wk  # noqa: E402

METRIC = "MLUPS (fluid-cell lattice updates per second) of the D3Q27 MRT pipe step"
NOMINAL_HBM_GBS = 7900.0      # GB300 HBM3e, nominal
BYTES_PER_UPDATE = {"f64": 432, "f32": 216, "f16s": 108, "bf16": 108}
LBM_STEPS_PER_STEP = 100


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5"])
    p.add_argument("--graph", type=int, default=None, help="steps per captured graph (0 = direct launches)")
    p.add_argument("--autotune", action="store_true", help="pick the step-kernel launch shape by timing")
    p.add_argument("--variant", type=int, default=None, help="force a step-kernel launch shape")
    p.add_argument("--precision", default="f32", choices=["f32", "f16s", "bf16", "f64"])
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def workload(name):
    return dict({"c2": Wk.C2, "c3": Wk.C3, "c4": Wk.C4, "c5": Wk.C5}[name])


def config_json(cfg, args, n_gpus, graph=0, tuned=None):
    out = {"workload": cfg["name"], "precision": args.precision, "wall": "halfway",
           "lbm_steps_per_step": LBM_STEPS_PER_STEP, "l2": "inputs larger than L2 (no flush)",
           "parallelism": "replicas x%d" % n_gpus, "graph_chunk": graph}
    if tuned is not None:
        out["launch_shape"] = {"variant": tuned[0], "us_per_step": tuned[1]}
    if args.workload == "c4":
        mem = Wk.ensemble_members(Wk.SEED, cfg["n"], cfg["radii"], cfg["u_star"])
        out.update({"members": cfg["n"], "radii": [m["R"] for m in mem], "nz": cfg["nz"],
                    "trigger_modes": [2]})
    else:
        out.update({"grid": [cfg["nx"], cfg["ny"], cfg["nz"]], "R": cfg["R"],
                    "stats_every": cfg["stats_every"], "mode_sections": cfg["n_sections"],
                    "n_theta": cfg["n_theta"], "trigger_modes": [m[0] for m in cfg["trigger_modes"]]})
    return out


# ---------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline): a bounded z-slab sample of the same pipe
# ---------------------------------------------------------------------------------------
def oracle_pipe(cfg):
    """The single pipe the oracle samples: the workload's pipe, or member 0 of the ensemble."""
    if "nx" in cfg:
        return dict(nx=cfg["nx"], ny=cfg["ny"], nz=cfg["nz"], R=cfg["R"], omega=cfg["omega"], h=cfg["h"],
                    period=cfg["period"], modes=cfg["trigger_modes"], t_end=cfg["t_trigger"], noise=cfg["noise"])
    mem = Wk.ensemble_members(Wk.SEED, cfg["n"], cfg["radii"], cfg["u_star"])[0]
    n = Wk.box_side(mem["R"])
    return dict(nx=n, ny=n, nz=cfg["nz"], R=mem["R"], omega=cfg["omega"], h=mem["h"], period=mem["period"],
                modes=[(2, 1.0, mem["phase"])], t_end=mem["t_end"], noise=Wk.C2["noise"])


def _oracle_sample(cfg, nz_sample, min_seconds, max_steps):
    from oracle import lbm as O
    pp = oracle_pipe(cfg)
    tr = O.Trigger(h=pp["h"], R=pp["R"], L=pp["nz"], period=pp["period"], modes=pp["modes"], t_end=pp["t_end"])
    run = O.Run(pp["nx"], pp["ny"], nz_sample, omega=pp["omega"], R=pp["R"], wall="halfway",
                g=(0.0, 0.0, pp["h"]), trigger=tr)
    run.init("loglaw", pp["noise"], Wk.SEED)
    n_fluid = int(run.fluid.sum())
    steps = 0
    t0 = time.perf_counter()
    while steps < max_steps:
        run.step(1)
        steps += 1
        if min_seconds > 0 and steps >= 2 and time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    return {"updates": n_fluid * steps, "seconds": dt, "steps": steps, "n_fluid": n_fluid,
            "shape": [pp["nx"], pp["ny"], nz_sample]}


def oracle_in_child(cfg_name, nz_sample, min_seconds, max_steps):
    """Runs the oracle sample in a fresh single-threaded interpreter (no GPU context)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._oracle_sample(bench.workload(%r), %d, %f, %d)))"
            % (ROOT, cfg_name, nz_sample, min_seconds, max_steps))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(args, cfg):
    nz_sample = 48
    res = oracle_in_child(args.workload, nz_sample, 10.0, 40)
    val = res["updates"] / res["seconds"] / 1e6
    return {"value": val, "unit": "MLUPS", "cores": 1, "kind": "oracle",
            "sample": "FP64 numpy oracle, %d steps of a %dx%dx%d z-slab of the same pipe (%d fluid cells), "
                      "one thread" % ((res["steps"],) + tuple(res["shape"]) + (res["n_fluid"],))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = workload(args.workload)
    nz_sample = 16
    for _ in range(args.warmup):
        oracle_in_child(args.workload, nz_sample, 0.0, 1)
    res = oracle_in_child(args.workload, nz_sample, 0.0, max(args.steps, 1))
    val = res["updates"] / res["seconds"] / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds"] / res["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_json(cfg, args, 1),
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                             "sample": "%d oracle steps of a %dx%dx%d z-slab per run" % (
                                 (res["steps"],) + tuple(res["shape"]))},
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(precision, workload_name):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", "k_step_%s_%s_traffic.txt" % (precision, workload_name))
    try:
        with open(path) as fh:
            for line in fh:
                if line.startswith("traffic_bytes_per_launch"):
                    return float(line.split(":")[1])
    except Exception:
        return None
    return None


def aggregate_ranks(ms, updates, dist=None, device="cpu"):
    """Whole-job timing across ranks: the slowest rank's time and the sum of every rank's
    lattice updates (each rank runs its own replica; no exchange on the data path)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, updates
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def build_single(lbm, cfg, args, stream, rank):
    grid = lbm.make_grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"], precision=args.precision, wall="halfway")
    trig = Wk.trigger_dict(h=cfg["h"], R=cfg["R"], nz=cfg["nz"], period=cfg["period"],
                           modes=cfg["trigger_modes"], t_end=cfg["t_trigger"])
    force = lbm.make_force(g=(0.0, 0.0, cfg["h"]), trigger=trig)
    L = lbm.Lattice(grid, lbm.lbm_relax(cfg["omega"]), force, stream=stream.cuda_stream)
    L.init("loglaw", noise_amp=cfg["noise"], seed=Wk.SEED + rank)
    lbm.lbm_stats_enable(L.ctx, cfg["stats_every"])
    return L


def build_ensemble(lbm, cfg, args, stream, rank):
    members = Wk.ensemble_members(Wk.SEED, cfg["n"], cfg["radii"], cfg["u_star"])
    grids, relaxes, forces = [], [], []
    for mem in members:
        R = mem["R"]
        n = Wk.box_side(R)
        grids.append(lbm.make_grid(n, n, cfg["nz"], R, precision=args.precision, wall="halfway"))
        relaxes.append(lbm.lbm_relax(cfg["omega"]))
        trig = Wk.trigger_dict(h=mem["h"], R=R, nz=cfg["nz"], period=mem["period"], modes=[(2, 1.0, mem["phase"])],
                               t_end=mem["t_end"])
        forces.append(lbm.make_force(g=(0.0, 0.0, mem["h"]), trigger=trig))
    L = lbm.Lattice(None, None, stream=stream.cuda_stream, ensemble=(grids, relaxes, forces))
    L.init("loglaw", noise_amp=cfg["noise"], seed=Wk.SEED + 1000 * rank)
    return L


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    cfg = workload(args.workload)
    ensemble = args.workload == "c4"
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, cfg)     # host-only child process, before heavy GPU use

    from paper_2405_12082_gb300 import lbm
    stream = torch.cuda.current_stream()
    L = (build_ensemble if ensemble else build_single)(lbm, cfg, args, stream, rank)
    info = L.info()
    n_members = info["n_members"]
    n_fluid = 0
    cells = []
    for m in range(n_members):
        L.select(m)
        mi = L.info()
        n_fluid += mi["n_fluid"]
        cells.append(mi["n_cells"])
    L.select(0)
    tuned = None
    if args.variant is not None:
        lbm.lbm_set_variant(L.ctx, args.variant)
        tuned = (args.variant, None)
    elif args.autotune or ensemble:
        tuned = lbm.lbm_autotune(L.ctx, 20)
    graph = args.graph if args.graph is not None else (LBM_STEPS_PER_STEP if ensemble else 0)
    if graph:
        lbm.lbm_set_graph(L.ctx, graph)
    if not ensemble:
        mcfg = lbm.make_modes_cfg(cfg["n_sections"], cfg["r_over_R"], cfg["n_theta"], cfg["n_modes"])
        E = torch.empty((cfg["n_sections"], len(cfg["r_over_R"]), cfg["n_modes"] + 1), dtype=torch.float64,
                        device="cuda")

    def one_step():
        lbm.lbm_step(L.ctx, LBM_STEPS_PER_STEP)
        if not ensemble:
            lbm.lbm_modes(L.ctx, mcfg, E)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.3)
    lbm.lbm_profile_enable(L.ctx, True)
    lbm.lbm_profile_read(L.ctx)
    launches0 = L.info()["launches"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kernel_ms, kernel_launches = lbm.lbm_profile_read(L.ctx)
    lbm.lbm_profile_enable(L.ctx, False)
    launches = L.info()["launches"] - launches0
    clk = clocks.stop()
    ms, updates = aggregate_ranks(ms, n_fluid * LBM_STEPS_PER_STEP * args.steps, dist, "cuda")
    value = updates / (ms * 1e-3) / 1e6

    # end to end through the C ABI with host buffers: upload the state from pinned host
    # memory, advance one bench step, read the results back to host memory (ring energies
    # and the velocity field; for the ensemble every member's velocity field)
    nbytes = info["population_bytes"]
    host_state = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    lbm.lbm_get_raw(L.ctx, host_state, nbytes)
    fdt = torch.float64 if args.precision == "f64" else torch.float32
    rho_h = [torch.empty(c, dtype=fdt, pin_memory=True) for c in cells]
    u_h = [torch.empty(3 * c, dtype=fdt, pin_memory=True) for c in cells]
    E_h = None if ensemble else np.empty((cfg["n_sections"], len(cfg["r_over_R"]), cfg["n_modes"] + 1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        lbm.lbm_set_raw(L.ctx, host_state, nbytes)
        lbm.lbm_step(L.ctx, LBM_STEPS_PER_STEP)
        if not ensemble:
            lbm.lbm_modes(L.ctx, mcfg, E_h)
        for m in range(n_members):
            L.select(m)
            lbm.lbm_moments(L.ctx, rho_h[m], u_h[m])
        L.select(0)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = n_fluid * LBM_STEPS_PER_STEP * max(args.e2e_steps, 1) * world / max(e2e_s, 1e-9) / 1e6
    d2h = sum(r.numel() * r.element_size() + u.numel() * u.element_size() for r, u in zip(rho_h, u_h))
    if E_h is not None:
        d2h += E_h.nbytes

    bad = 0.0
    for m in range(n_members):
        L.select(m)
        bad += lbm.lbm_reduce(L.ctx)[4]
    L.close()
    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = measured_peak()
    avg_kernel_s = (kernel_ms / kernel_launches) * 1e-3 if kernel_launches else None
    bpu = BYTES_PER_UPDATE[args.precision]
    achieved = bpu * n_fluid / avg_kernel_s / 1e9 if avg_kernel_s else None
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "f64" else "f32",
        "storage": args.precision, "data": "synthetic (seeded log-law + noise, paper-shaped pipe)",
        "config": config_json(cfg, args, world, graph, tuned),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": profiled_traffic(args.precision, args.workload),
                     "kernel": "k_step", "bytes_per_update": bpu, "peak_kind": peak_kind,
                     "avg_kernel_us": avg_kernel_s * 1e6 if avg_kernel_s else None,
                     "frac_of_nominal": achieved / NOMINAL_HBM_GBS if achieved else None,
                     "nominal_gbs": NOMINAL_HBM_GBS},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "n_fluid_cells": n_fluid,
        "all_cell_mlups": value * sum(cells) / n_fluid,
        "nonfinite_cells": bad,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_adjoint_bench(args):
    """Forward MLUPS and the adjoint/forward time ratio on the 52 x 52 x 256, R = 24 pipe
    (T = 2000 steps, FP32, per-cell axial acceleration): the adjoint call runs its own
    forward pass with checkpoints, recomputes every segment and sweeps backwards."""
    import numpy as np
    import torch
    from paper_2405_12082_gb300 import lbm
    cfg = workload("c5")
    prec = args.precision
    dt = torch.float64 if prec == "f64" else torch.float32
    gz = torch.full((cfg["nz"], cfg["ny"], cfg["nx"]), cfg["gz"], dtype=dt, device="cuda")
    grid = lbm.make_grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"], precision=prec, wall="halfway")
    stream = torch.cuda.current_stream()
    L = lbm.Lattice(grid, lbm.lbm_relax(cfg["omega"]), lbm.make_force(gz_field=gz), stream=stream.cuda_stream)
    L.init("rest")
    n_fluid = L.info()["n_fluid"]
    T = cfg["T"]
    L.step(200)
    dgz = torch.zeros_like(gz, dtype=torch.float64)
    lbm.lbm_adjoint(L.ctx, 50, lbm.LBM_J_UBULK, 0, dgz)      # warm-up of the adjoint path
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fwd = []
    for _ in range(max(args.steps, 1)):
        e0.record(stream)
        L.step(T)
        e1.record(stream)
        torch.cuda.synchronize()
        fwd.append(e0.elapsed_time(e1))
    adj = []
    for _ in range(max(args.steps, 1)):
        e0.record(stream)
        J, dw = lbm.lbm_adjoint(L.ctx, T, lbm.LBM_J_UBULK, 0, dgz)
        e1.record(stream)
        torch.cuda.synchronize()
        adj.append(e0.elapsed_time(e1))
    # the same call with one segment: the forward pass stores the moments of every step
    # (T x 9 values per stored cell) and nothing is recomputed; timed where memory allows
    store_all = None
    es = 8 if prec == "f64" else 4
    mom_bytes = T * 9 * L.info()["n_cells"] * es
    if torch.cuda.mem_get_info()[0] > 2 * mom_bytes:
        sa = []
        for _ in range(max(args.steps, 1)):
            e0.record(stream)
            lbm.lbm_adjoint(L.ctx, T, lbm.LBM_J_UBULK, T, dgz)
            e1.record(stream)
            torch.cuda.synchronize()
            sa.append(e0.elapsed_time(e1))
        store_all = {"adjoint_call_ms": min(sa), "moment_bytes": mom_bytes}
    L.close()
    f_ms, a_ms = min(fwd), min(adj)
    if store_all is not None:
        store_all["reverse_over_forward"] = (store_all["adjoint_call_ms"] - f_ms) / f_ms
    line = {"metric": METRIC + "; adjoint/forward time ratio", "value": n_fluid * T / (f_ms * 1e-3) / 1e6,
            "unit": "MLUPS", "n_gpus": 1, "steps": len(fwd), "warmup": 1, "ms_per_step": f_ms / T,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "f64" else "f32", "storage": prec, "data": "synthetic (rest start)",
            "config": {"workload": cfg["name"], "grid": [cfg["nx"], cfg["ny"], cfg["nz"]], "R": cfg["R"],
                       "T": T, "checkpoints": "every ceil(sqrt(T)) steps", "objective": "bulk velocity"},
            "adjoint": {"forward_ms": f_ms, "adjoint_call_ms": a_ms,
                        "reverse_over_forward": (a_ms - f_ms) / f_ms, "total_over_forward": a_ms / f_ms,
                        "J": J, "dJ_domega": dw, "store_all_steps": store_all}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c5":
        return run_adjoint_bench(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
