"""Throughput of the fused D3Q27 MRT pipe step on one GB300 (JSON line on stdout).

Workload (default): the R = 96 pipe, 196 x 196 x 1152 cells (33.4 M fluid cells), FP32
shifted populations, Re_tau = 181.3 parameters, log-law start with 5 % Gaussian noise,
the four-mode trigger force active (the flow is still developing inside the timed
steps), FP64 statistics every 100 steps and the 16-section azimuthal mode analysis once
per bench step.  One bench step = 100 lattice steps (one of them with the fused
statistics accumulation) + one mode analysis, i.e. every row of the hot path.  The
population array (4.8 GB) is larger than L2, so no flush is needed between steps.

The same line also carries, measured in the same run:
  precisions  the same bench step with F16S and BF16 storage (FP32 collision);
  adjoint     the adjoint pipe 52 x 52 x 256 (T = 2000, sqrt(T) checkpoints): forward
              time, adjoint-call time and their ratio;
  cpu_baseline  the FP64 oracle on a z-slab of the same pipe, on one thread and on
              every host core (one single-threaded process per core), CPU model named.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c3|c2|c4|c5] [--precision f32|f16s|bf16|f64] [--no-extras]

Under torchrun (N > 1) every rank runs its own replica of the pipe on its own GPU
(the path has no exchange step); rank 0 prints the aggregate.
`--impl reference` times the FP64 oracle on the host cores instead.
"""
import argparse
import hashlib
import json
import os
import platform
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
    p.add_argument("--workload", default="c3", choices=["c2", "c3", "c4", "c5"])
    p.add_argument("--graph", type=int, default=None, help="steps per captured graph (0 = direct launches)")
    p.add_argument("--autotune", action="store_true", help="pick the step-kernel launch shape by timing")
    p.add_argument("--variant", type=int, default=None, help="force a step-kernel launch shape")
    p.add_argument("--precision", default="f32", choices=["f32", "f16s", "bf16", "f64"])
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the 16-bit storage and adjoint measurements")
    return p.parse_args()


def workload(name):
    return dict({"c2": Wk.C2, "c3": Wk.C3, "c4": Wk.C4, "c5": Wk.C5}[name])


def config_json(cfg, args, n_gpus, graph=0, tuned=None):
    out = {"workload": cfg["name"], "precision": args.precision, "wall": "halfway",
           "lbm_steps_per_step": LBM_STEPS_PER_STEP, "l2": "inputs larger than L2 (no flush)",
           "parallelism": "replicas x%d" % n_gpus, "graph_chunk": graph}
    if tuned is not None:
        # the shapes themselves are the line's launch_shape key (even and odd steps)
        out["launch_shape"] = {"chosen_by": "--variant" if tuned[1] is None else "lbm_autotune",
                               "mean_us_per_step": tuned[1]}
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


def _child_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
                CUDA_VISIBLE_DEVICES="")


def _child_cmd(cfg_name, nz_sample, min_seconds, max_steps):
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench._oracle_sample(bench.workload(%r), %d, %f, %d)))"
            % (ROOT, cfg_name, nz_sample, min_seconds, max_steps))
    return [sys.executable, "-c", code]


def oracle_in_children(cfg_name, nz_sample, min_seconds, max_steps, n_proc=1):
    """Runs the oracle sample in n_proc fresh single-threaded interpreters at once (no GPU
    context in any of them).  Each child times only its own step loop; the aggregate rate
    is the sum of the children's updates over the longest child time."""
    procs = [subprocess.Popen(_child_cmd(cfg_name, nz_sample, min_seconds, max_steps), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=_child_env(), cwd=ROOT)
             for _ in range(n_proc)]
    res = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("oracle sample failed: " + err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    return {"updates": sum(r["updates"] for r in res), "seconds": max(r["seconds"] for r in res),
            "steps": min(r["steps"] for r in res), "n_fluid": res[0]["n_fluid"], "shape": res[0]["shape"],
            "n_proc": n_proc}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model():
    """CPU model of the host as the OS reports it (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                return v.strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            if k.strip() in ("model name", "CPU part") and v.strip():
                return v.strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


# z-slab thickness of the oracle sample per workload (bounded CPU work per step)
SLAB_NZ = {"c2": 16, "c3": 8, "c4": 16, "c5": 16}


def slab_text(res):
    return "%dx%dx%d z-slab (%d fluid cells) of the same pipe" % (tuple(res["shape"]) + (res["n_fluid"],))


def cpu_baseline(args, cfg):
    """The FP64 oracle timed on the host cores: one thread, then one single-threaded
    process per core at once (about 10 s each)."""
    nz = SLAB_NZ[args.workload]
    one = oracle_in_children(args.workload, nz, 10.0, 60, 1)
    n = host_cores()
    allc = oracle_in_children(args.workload, nz, 10.0, 60, n)
    v1 = one["updates"] / one["seconds"] / 1e6
    vn = allc["updates"] / allc["seconds"] / 1e6
    return {"value": vn, "unit": "MLUPS", "cores": n, "kind": "oracle",
            "sample": "FP64 numpy oracle, %d concurrent single-threaded processes, each >= %d steps of a %s"
                      % (n, allc["steps"], slab_text(allc)),
            "single_thread": {"value": v1, "cores": 1, "steps": one["steps"]},
            "cpu_model": cpu_model(), "nproc": n}


def reference_config(cfg, args, res):
    out = config_json(cfg, args, 1)
    out["workload"] = "FP64 oracle on a " + slab_text(res) + " of: " + cfg["name"]
    out["timed_sample"] = {"grid": res["shape"], "n_fluid": res["n_fluid"], "processes": res["n_proc"],
                           "of_workload": cfg["name"]}
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on every host core (one
    single-threaded process per core, each stepping its own z-slab of the pipe)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = workload(args.workload)
    nz = SLAB_NZ[args.workload]
    n = host_cores()
    if args.warmup > 0:
        oracle_in_children(args.workload, nz, 0.0, 1, 1)
    res = oracle_in_children(args.workload, nz, 0.0, max(args.steps, 1), n)
    val = res["updates"] / res["seconds"] / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * res["seconds"] / res["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": reference_config(cfg, args, res),
            "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": n, "kind": "oracle",
                             "sample": "%d concurrent single-threaded processes, %d oracle steps each of a %s"
                                       % (n, res["steps"], slab_text(res)),
                             "cpu_model": cpu_model(), "nproc": n},
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


# the files that define the step kernel: a traffic figure counts only while they are
# unchanged since the ncu capture that produced it
KERNEL_SOURCES = ("lbm_device.cuh", "lbm_kernels.cuh", "lbm_staged.cuh", "lbm_internal.h", "lbm_f32.cu",
                  "lbm_f64.cu", "lbm_f16s.cu", "lbm_bf16.cu")


def kernel_sources_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2405_12082_gb300", "csrc")
    for name in KERNEL_SOURCES:
        path = os.path.join(csrc, name)
        if os.path.exists(path):
            h.update(name.encode())
            h.update(open(path, "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(precision, workload_name):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, or None
    when there is none or the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "k_step_%s_%s_traffic.txt" % (precision, workload_name))
    vals = {}
    try:
        with open(path) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, _, v = line.partition(":")
                    vals[k.strip()] = v.strip()
    except Exception:
        return None
    if vals.get("kernel_sources_sha16") != kernel_sources_sha():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except Exception:
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
    shapes = L.info()             # the launch shapes the timed steps run (after any tuning)
    shapes = {"even": shapes["variant"], "odd": shapes["variant_odd"]}
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
    def e2e_step():
        lbm.lbm_set_raw(L.ctx, host_state, nbytes)
        lbm.lbm_step(L.ctx, LBM_STEPS_PER_STEP)
        if not ensemble:
            lbm.lbm_modes(L.ctx, mcfg, E_h)
        for m in range(n_members):
            L.select(m)
            lbm.lbm_moments(L.ctx, rho_h[m], u_h[m])
        L.select(0)

    for _ in range(2):            # untimed: staging buffers, first touch of the pinned pages
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms, e2e_updates = aggregate_ranks((time.perf_counter() - t0) * 1e3,
                                          n_fluid * LBM_STEPS_PER_STEP * max(args.e2e_steps, 1), dist, "cuda")
    e2e_val = e2e_updates / max(e2e_ms * 1e-3, 1e-12) / 1e6
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

    extras = {}
    if world == 1 and not args.no_extras and not ensemble:
        reps = max(1, min(args.steps, 10))
        extras["precisions"] = {p: measure_precision(lbm, cfg, args, p, reps, 2)
                                for p in ("f32", "f16s", "bf16") if p != args.precision}
        extras["adjoint"] = measure_adjoint(lbm, min(reps, 3))

    peak, peak_kind = measured_peak()
    extras["alu_probe"] = alu_probe(lbm, torch, peak)
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
                     "kernel_sources_sha16": kernel_sources_sha(),
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
        "launch_shape": shapes,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def alu_probe(lbm, torch, hbm_gbs):
    """The instruction side of the roofline: the measured FP32 FMA rates of this GPU and, at
    that issue rate, how many thread instructions one fluid-cell update may take for the step
    to run at the measured copy bandwidth with each storage (216 B and 108 B per update)."""
    try:
        r = lbm.lbm_probe_fp32(torch.cuda.current_stream().cuda_stream)
    except lbm.LbmError as e:
        return {"error": str(e)}
    smsp = 4 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    thread_inst_per_s = r["warp_ffma_per_s_per_smsp"] * smsp * 32
    r["thread_inst_slots_per_update_at_hbm_roof"] = {
        prec: thread_inst_per_s / (hbm_gbs * 1e9 / b) for prec, b in (("f32", 216), ("f16s", 108), ("bf16", 108))}
    return r


def measure_precision(lbm, cfg, args, precision, steps, warmup):
    """The bench step of the workload with another storage precision: G fluid updates/s and
    the step kernel's mean launch time and roofline fraction (CUDA events)."""
    import torch
    a = argparse.Namespace(**vars(args))
    a.precision = precision
    stream = torch.cuda.current_stream()
    L = build_single(lbm, cfg, a, stream, 0)
    n_fluid = L.info()["n_fluid"]
    mcfg = lbm.make_modes_cfg(cfg["n_sections"], cfg["r_over_R"], cfg["n_theta"], cfg["n_modes"])
    E = torch.empty((cfg["n_sections"], len(cfg["r_over_R"]), cfg["n_modes"] + 1), dtype=torch.float64,
                    device="cuda")

    def one_step():
        lbm.lbm_step(L.ctx, LBM_STEPS_PER_STEP)
        lbm.lbm_modes(L.ctx, mcfg, E)

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    lbm.lbm_profile_enable(L.ctx, True)
    lbm.lbm_profile_read(L.ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kms, kn = lbm.lbm_profile_read(L.ctx)
    lbm.lbm_profile_enable(L.ctx, False)
    bad = lbm.lbm_reduce(L.ctx)[4]
    variant = {"even": L.info()["variant"], "odd": L.info()["variant_odd"]}
    L.close()
    peak, _ = measured_peak()
    bpu = BYTES_PER_UPDATE[precision]
    avg_s = (kms / kn) * 1e-3 if kn else None
    achieved = bpu * n_fluid / avg_s / 1e9 if avg_s else None
    return {"value": n_fluid * LBM_STEPS_PER_STEP * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "steps": steps,
            "ms_per_step": ms / steps, "bytes_per_update": bpu, "avg_kernel_us": avg_s * 1e6 if avg_s else None,
            "achieved_gbs": achieved, "frac": achieved / peak if achieved else None, "launch_shape": variant,
            "nonfinite_cells": bad}


def measure_adjoint(lbm, reps, precision="f32", store_all=True):
    """Forward and adjoint-call times on the adjoint pipe (52 x 52 x 256, R = 24, T = 2000,
    per-cell axial acceleration, rest start advanced 200 steps): the adjoint call runs its
    own forward pass with checkpoints every ceil(sqrt(T)) steps, recomputes each segment
    and sweeps backwards.  Best of `reps` calls each."""
    import torch
    cfg = workload("c5")
    dt = torch.float64 if precision == "f64" else torch.float32
    gz = torch.full((cfg["nz"], cfg["ny"], cfg["nx"]), cfg["gz"], dtype=dt, device="cuda")
    grid = lbm.make_grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"], precision=precision, wall="halfway")
    stream = torch.cuda.current_stream()
    L = lbm.Lattice(grid, lbm.lbm_relax(cfg["omega"]), lbm.make_force(gz_field=gz), stream=stream.cuda_stream)
    L._keep.append(gz)
    L.init("rest")
    n_fluid = L.info()["n_fluid"]
    T = cfg["T"]
    L.step(200)
    dgz = torch.zeros_like(gz, dtype=torch.float64)
    lbm.lbm_adjoint(L.ctx, 50, lbm.LBM_J_UBULK, 0, dgz)      # warm-up of the adjoint path
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        best = None
        for _ in range(max(reps, 1)):
            e0.record(stream)
            r = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best, r

    f_ms, _ = timed(lambda: L.step(T))
    a_ms, (J, dw) = timed(lambda: lbm.lbm_adjoint(L.ctx, T, lbm.LBM_J_UBULK, 0, dgz))
    sa = None
    es = 8 if precision == "f64" else 4
    mom_bytes = T * 9 * L.info()["n_cells"] * es
    if store_all and torch.cuda.mem_get_info()[0] > 2 * mom_bytes:
        s_ms, _ = timed(lambda: lbm.lbm_adjoint(L.ctx, T, lbm.LBM_J_UBULK, T, dgz))
        sa = {"adjoint_call_ms": s_ms, "moment_bytes": mom_bytes, "reverse_over_forward": (s_ms - f_ms) / f_ms}
    L.close()
    return {"workload": cfg["name"], "T": T, "precision": precision, "checkpoints": "every ceil(sqrt(T)) steps",
            "objective": "bulk velocity", "forward_ms": f_ms, "forward_mlups": n_fluid * T / (f_ms * 1e-3) / 1e6,
            "adjoint_call_ms": a_ms, "reverse_over_forward": (a_ms - f_ms) / f_ms,
            "total_over_forward": a_ms / f_ms, "J": J, "dJ_domega": dw, "store_all_steps": sa}


def run_adjoint_bench(args):
    """Forward MLUPS and the adjoint/forward time ratio on the 52 x 52 x 256, R = 24 pipe
    (T = 2000 steps, per-cell axial acceleration): see measure_adjoint."""
    from paper_2405_12082_gb300 import lbm
    prec = args.precision
    adj = measure_adjoint(lbm, max(args.steps, 1), prec)
    cfg = workload("c5")
    line = {"metric": METRIC + "; adjoint/forward time ratio", "value": adj["forward_mlups"],
            "unit": "MLUPS", "n_gpus": 1, "steps": max(args.steps, 1), "warmup": 1,
            "ms_per_step": adj["forward_ms"] / adj["T"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "f64" else "f32", "storage": prec, "data": "synthetic (rest start)",
            "config": {"workload": cfg["name"], "grid": [cfg["nx"], cfg["ny"], cfg["nz"]], "R": cfg["R"],
                       "T": adj["T"], "checkpoints": adj["checkpoints"], "objective": adj["objective"]},
            "adjoint": adj}
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
