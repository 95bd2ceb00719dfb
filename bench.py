#!/usr/bin/env python
"""Throughput of the differentiable XPBD step on one GB300 (or N independent replicas).

One bench step = the whole hot path over the 2950 x 2950 cloth draped on a sphere
(8,702,500 vertices, 34,792,302 distance + 17,387,304 bending constraints, 60 steps of
15 colored Gauss-Seidel iterations): forward simulation with per-step checkpoints, the
keyframe loss at steps 20/40/60 with its seeds, and the full reverse sweep giving float64
gradients for every compliance, x0, v0, the 60x3 per-step global force, the per-vertex
force field and the sphere parameters.

metric: fwd+adjoint constraint-updates/s = 2 * m * iters * steps / time per bench step
(each constraint update of the forward and each reverse (VJP) update of the adjoint counts
once; the in-adjoint replay is part of the adjoint's cost, not counted as extra units).

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2301_01396_gb300 import scenes  # noqa: E402

METRIC = "fwd+adjoint constraint-updates/s"
UNIT = "constraint-updates/s"
KEYFRAMES = (20, 40, 60)
GRID = 2950
TILE = 32

# Algorithmic bytes of each kernel class come from the library (xpbd_profile_read: its byte
# model counts records, multipliers, tapes and one read plus one write per vertex per launch).


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--grid", type=int, default=GRID, help="cloth side (default: the 2950^2 workload)")
    ap.add_argument("--coloring", choices=("tiled", "pattern"), default="tiled",
                    help="constraint coloring of the cloth (tiled: square vertex blocks in 4 classes)")
    ap.add_argument("--tile", type=int, default=TILE, help="tile side of the tiled coloring")
    ap.add_argument("--checkpoint-stride", type=int, default=0,
                    help="store the state only every K steps and recompute the rest in the reverse sweep "
                         "(0: every step)")
    ap.add_argument("--keyframe-scale", action="store_true",
                    help="the paper's keyframe-example scale instead of the default workload: 900 steps x 20 "
                         "iterations on a 90x90 cloth with a force per vertex per step (21.9M controls)")
    ap.add_argument("--implicit", action="store_true",
                    help="time the paper's implicit adjoint next to the discrete one on the 256^2 ground cloth")
    ap.add_argument("--implicit-grid", type=int, default=256)
    ap.add_argument("--implicit-precond", choices=("multigrid", "multigrid-points", "jacobi"), default="multigrid",
                    help="CG preconditioner of the implicit adjoint: grid multigrid with diagonal-line smoothing "
                         "on the finest level (the ground cloth folds freely along its diagonals), with point "
                         "smoothing only, or 3x3 block Jacobi")
    ap.add_argument("--mg-sweeps", type=int, default=1)
    ap.add_argument("--cg-tol", type=float, default=1e-6)
    ap.add_argument("--material", choices=("tets", "tets-coupled", "membrane"), default=None,
                    help="material-estimation workloads: the 32^3 tet block (one constraint at a time, or each "
                         "tet's pair by a 2x2 solve) with 100 materials, or a 256^2 orthotropic StVK membrane cloth")
    ap.add_argument("--material-tile", type=int, default=8, help="tile side of the membrane cloth's coloring")
    ap.add_argument("--material-grid", type=int, default=256, help="side of the membrane cloth")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-window", type=int, default=160)
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--sim-steps", type=int, default=0,
                    help="profiling aid: shorter horizon (same per-step kernel mix); not a bench value")
    ap.add_argument("--iters", type=int, default=0, help="profiling aid: fewer iterations; not a bench value")
    ap.add_argument("--serving", action="store_true",
                    help="serving stream instead of the default workload: p50/p99 latency and steps/s, "
                         "continuous batching vs one request at a time")
    ap.add_argument("--serving-requests", type=int, default=120)
    ap.add_argument("--serving-load", type=float, default=1.0,
                    help="arrival rate as a multiple of the one-at-a-time service rate")
    ap.add_argument("--serving-slots", type=int, default=64)
    ap.add_argument("--serving-ticks", type=int, default=32, help="ticks per server batch (one launch)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(ws):
    if ws > 1:
        import torch.distributed as td
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        td.init_process_group(backend=backend)


def barrier(ws):
    if ws > 1:
        import torch.distributed as td
        td.barrier()


def max_over_ranks(ws, v: float) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as td
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ws: int, units_per_rank: float, ms_local: float):
    """Whole-job rate of N independent replicas: every rank processed `units_per_rank`
    units and the job took as long as its slowest rank.  Returns (units/s, ms)."""
    ms_max = max_over_ranks(ws, ms_local)
    return ws * units_per_rank / (ms_max / 1e3), ms_max


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.dev = device_index

    def start(self):
        sel = []
        try:
            import torch
            u = getattr(torch.cuda.get_device_properties(self.dev), "uuid", None)
            if u is not None:
                sel = ["-i", "GPU-" + str(u)]
        except Exception:
            sel = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", *sel], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power) if power else None}


# ----------------------------------------------------------------------------- workload

def workload(grid: int, coloring: str = "tiled", tile: int = TILE):
    t0 = time.time()
    sc = scenes.sphere_cloth(grid, coloring=coloring, tile=tile)
    return sc, time.time() - t0


def cpu_window_scene(nw: int, steps: int, grid: int = GRID):
    """A nw x nw window of the grid x grid cloth: same spacing, vertex mass, constraint
    types and compliance law, centred over the sphere; the oracle's bounded sample."""
    size = (nw - 1) / (grid - 1)
    g = scenes.cloth_grid(nw, size, vertex_mass=2.56 / grid ** 2, diagonals="both", bending=True, pins=(),
                          origin=(0.5 - size / 2, 0.5 - size / 2))
    rng = np.random.default_rng(4)
    alpha = scenes.lognormal_cloth_compliance(rng, g["dist_idx"].shape[0], g["bend_idx"].shape[0])
    return scenes._cloth_scene(g, alpha, dt=1.0 / 60.0, steps=steps, iters=15,
                               collider_flags=scenes.COLLIDE_SPHERE, sphere=(0.5, -0.35, 0.5, 0.3),
                               contact_compliance=1e-8, name=f"window_{nw}")


def run_cpu_oracle(nw: int, steps: int) -> dict:
    """Time the FP64 oracle (as it stands) on a window of the workload: forward + reverse."""
    import oracle
    sc = cpu_window_scene(nw, steps)
    t0 = time.perf_counter()
    xs, _ = oracle.forward(sc)
    t1 = time.perf_counter()
    oracle.adjoint(sc, {steps: xs[-1] - sc.x0})
    t2 = time.perf_counter()
    units = 2 * sc.m * sc.iters * steps
    return {"value": units / (t2 - t0), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{nw}x{nw} window of the {GRID}x{GRID} cloth (same spacing, masses, constraint types "
                      f"and compliance law; {sc.m} constraints), {steps} steps x 15 iterations, forward + "
                      f"reverse sweep, FP64; forward {t1 - t0:.2f} s, reverse {t2 - t1:.2f} s"}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_for(cls: str, units_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the kernel
    source that is built now; otherwise None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    e = d.get("classes", {}).get(cls)
    if not e or d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return float(e["dram_bytes_per_unit"]) * units_per_launch


KERNEL_SOURCES = ("csrc/xpbd_phase.cu", "csrc/xpbd_kernels.cu", "csrc/xpbd_elems.cuh", "csrc/xpbd_math.cuh",
                  "csrc/xpbd_kernels.cuh", "build.py")


def kernel_source_hash() -> str:
    """Fingerprint of the sources and build flags of the constraint kernels."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2301_01396_gb300", f), "rb").read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------- checkpoints

def new_checkpoints(solver, N, stride, dev):
    """Dense (every step) or sparse (every `stride`-th step and the last) checkpoint buffer."""
    import torch
    from paper_2301_01396_gb300 import binding
    if not stride:
        return solver.new_checkpoints(N, dev)
    return torch.empty((binding.sparse_slots(N, stride), 2, solver.V, 4), dtype=torch.float32, device=dev)


def ck_index(N, stride, step):
    """Index of a step's state in the checkpoint buffer."""
    from paper_2301_01396_gb300 import binding
    if not stride:
        return step
    s = binding.sparse_slot(N, stride, step)
    if s < 0:
        raise SystemExit(f"keyframe step {step} is not stored with --checkpoint-stride {stride}")
    return s


def run_forward(solver, p, N, I, x0, v0, ck, stride):
    if stride:
        solver.forward_sparse(p, N, I, x0, v0, stride, checkpoints=ck)
    else:
        solver.forward(p, N, I, x0, v0, checkpoints=ck)


# ----------------------------------------------------------------------------- our arm

def run_ours(args, ws, rank, local):
    import torch
    from paper_2301_01396_gb300 import binding

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc, t_gen = workload(args.grid, args.coloring, args.tile)
    if args.sim_steps:
        sc.steps = args.sim_steps
        sc.f_global = sc.f_global[:args.sim_steps]
    if args.iters:
        sc.iters = args.iters
    N, I = sc.steps, sc.iters
    keys = tuple(k for k in KEYFRAMES if k <= N) or (N,)
    t0 = time.time()
    solver = binding.Solver.from_scene(sc)
    t_create = time.time() - t0
    x0 = torch.as_tensor(sc.x0.astype(np.float32), device=dev)
    v0 = torch.as_tensor(sc.v0.astype(np.float32), device=dev)
    p_true = binding.params_from_scene(sc, device=dev)
    K = args.checkpoint_stride
    ck = new_checkpoints(solver, N, K, dev)
    ckk = {k: ck_index(N, K, k) for k in keys}   # keyframe -> checkpoint index

    # keyframe targets from the driven simulation; the optimisation starts from zero forces
    run_forward(solver, p_true, N, I, x0, v0, ck, K)
    targets = {k: solver.read_state(ck, ckk[k])[0].clone() for k in keys}
    params = binding.Params(dt=p_true.dt, compliance=p_true.compliance, gravity=p_true.gravity,
                            f_global=torch.zeros((N, 3), dtype=torch.float32, device=dev),
                            f_vertex=torch.zeros((sc.V, 3), dtype=torch.float32, device=dev),
                            collider_flags=p_true.collider_flags, plane_h=p_true.plane_h, sphere=p_true.sphere,
                            contact_compliance=p_true.contact_compliance, thickness=p_true.thickness)
    grads = {k: torch.empty(s, dtype=torch.float64, device=dev)
             for k, s in dict(compliance=(sc.m,), x0=(sc.V, 3), v0=(sc.V, 3), f_global=(N, 3),
                              f_vertex=(sc.V, 3), collider=(5,)).items()}
    loss_box = {}

    def step():
        run_forward(solver, params, N, I, x0, v0, ck, K)
        loss, seeds = solver.loss(ck, {ckk[k]: targets[k] for k in keys})
        solver.adjoint(params, N, I, ck, {k: seeds[i] for i, k in enumerate(keys)}, out=grads, stride=K or None)
        loss_box["loss"] = loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    solver.sync_status()

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    solver.profile(True)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    stats = solver.profile_read()
    solver.profile(False)
    solver.sync_status()
    ms = e0.elapsed_time(e1) / args.steps
    units = 2 * sc.m * I * N
    value, ms_max = replica_rate(ws, units, ms)

    # dominant kernel class and its roofline: algorithmic bytes per launch (the library's
    # byte model: records, multipliers, tapes, one read and one write per vertex per launch)
    # over the class's mean CUDA-event launch time
    timed = {k: v for k, v in stats.items() if v["timed_launches"] > 0 and v["alg_bytes"] > 0}
    dom = max(timed, key=lambda k: timed[k]["ms"])
    d = timed[dom]
    avg_ms = d["ms"] / d["timed_launches"]
    upl = d["units"] / d["launches"]
    bpl = d["alg_bytes"] / d["launches"]
    achieved = bpl / (avg_ms / 1e3) / 1e9
    peak, peak_kind = measured_peak()
    tr = traffic_for(dom, upl)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None if tr is None else round(tr),
                "kernel": dom, "launch_avg_ms": round(avg_ms, 4), "units_per_launch": round(upl),
                "bytes_per_unit": round(bpl / upl, 2), "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": round(bpl)}
    launches = int(sum(v["launches"] for v in stats.values()))
    breakdown = {k: round(v["ms"] / args.steps, 2) for k, v in sorted(stats.items(), key=lambda kv: -kv[1]["ms"])
                 if v["ms"] > 0}
    # per class: algorithmic bytes per constraint (or vertex) update and the rate they
    # were moved at over the class's CUDA-event time
    class_bytes = {k: {"bytes_per_unit": round(v["alg_bytes"] / v["units"], 2),
                       "gbs": round(v["alg_bytes"] * v["timed_launches"] / v["launches"] / (v["ms"] / 1e3) / 1e9, 1)}
                   for k, v in timed.items() if v["units"] > 0}
    fwd_ms = sum(v["ms"] for k, v in stats.items() if k.startswith("fwd_") or k in ("predict", "velocity")) / args.steps
    plan = solver.exec_info()
    all_bytes = sum(v["alg_bytes"] for v in stats.values()) / args.steps
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (f64 gradient reductions)", "data": "synthetic",
        "config": {"workload": f"sphere_cloth_{args.grid}x{args.grid}: {sc.V} vertices, {sc.n_dist} distance + "
                               f"{sc.n_bend} bending constraints, {N} steps x {I} iterations, dt=1/60, sphere "
                               f"collider, keyframe loss at {list(keys)}, gradients for compliance/x0/v0/"
                               f"f_global/f_vertex/sphere",
                   "V": sc.V, "m": sc.m, "sim_steps": N, "iters": I, "colors": sc.n_colors,
                   "coloring": args.coloring + (f" {args.tile}x{args.tile}" if args.coloring == "tiled" else ""),
                   "launches_per_iteration": plan["launches_per_iteration"], "phase_kernels": plan["phases"],
                   "l2": "inputs larger than L2 (vertex state 139 MB, records 1.1 GB, tapes 36 GB)",
                   "parallelism": f"replicas x{ws}",
                   "checkpoints": ({"stride": K, "states_stored": int(ck.shape[0]), "recomputed_states": K - 1,
                                    "bytes": int(ck.numel() * 4 + max(K - 1, 0) * 32 * sc.V)} if K else
                                   {"stride": 1, "states_stored": N + 1, "bytes": int(ck.numel() * 4)}),
                   **({"profiling_override": f"sim_steps={N} iters={I} (not a bench value)"}
                      if (args.sim_steps or args.iters) else {})},
        "roofline": roofline,
        "clocks": clk,
        "gpu_launches": launches,
        "breakdown_ms_per_step": breakdown,
        "class_bytes": class_bytes,
        "forward_ms_per_step": round(fwd_ms, 2),
        "adjoint_ms_per_step": round(ms - fwd_ms, 2),
        "algorithmic_gb_per_step": round(all_bytes / 1e9, 1),
        "loss": float(loss_box["loss"].item()),
        "setup_s": {"scene": round(t_gen, 1), "create": round(t_create, 1)},
    }

    if not args.no_e2e:
        result["e2e"] = run_e2e(args, sc, solver, params, targets, keys, dev, ws)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = run_cpu_oracle(args.cpu_window, args.cpu_steps)
    return result


def run_e2e(args, sc, solver, params, targets, keys, dev, ws):
    """Same metric through the public API with host buffers: every step copies its inputs
    host->device from pinned memory and the gradients and loss device->host."""
    import torch
    from paper_2301_01396_gb300 import binding
    N, I = sc.steps, sc.iters
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).pin_memory()
    h_x0, h_v0 = pin(sc.x0), pin(sc.v0)
    h_comp = pin(sc.compliance)
    h_fg, h_fv = pin(np.zeros((N, 3))), pin(np.zeros((sc.V, 3)))
    h_tg = pin(np.stack([targets[k].cpu().numpy() for k in keys]))
    shapes = dict(compliance=(sc.m,), x0=(sc.V, 3), v0=(sc.V, 3), f_global=(N, 3), f_vertex=(sc.V, 3), collider=(5,))
    h_out = {k: torch.empty(s, dtype=torch.float64).pin_memory() for k, s in shapes.items()}
    h_loss = torch.empty(1, dtype=torch.float64).pin_memory()
    K = args.checkpoint_stride
    ck = new_checkpoints(solver, N, K, dev)
    d_out = {k: torch.empty(s, dtype=torch.float64, device=dev) for k, s in shapes.items()}
    h2d = sum(t.numel() * t.element_size() for t in (h_x0, h_v0, h_comp, h_fg, h_fv, h_tg))
    d2h = sum(t.numel() * t.element_size() for t in h_out.values()) + 8

    def step():
        x0 = h_x0.to(dev, non_blocking=True)
        v0 = h_v0.to(dev, non_blocking=True)
        p = binding.Params(dt=params.dt, compliance=h_comp.to(dev, non_blocking=True), gravity=params.gravity,
                           f_global=h_fg.to(dev, non_blocking=True), f_vertex=h_fv.to(dev, non_blocking=True),
                           collider_flags=params.collider_flags, plane_h=params.plane_h, sphere=params.sphere,
                           contact_compliance=params.contact_compliance, thickness=params.thickness)
        tg = h_tg.to(dev, non_blocking=True)
        run_forward(solver, p, N, I, x0, v0, ck, K)
        loss, seeds = solver.loss(ck, {ck_index(N, K, k): tg[i] for i, k in enumerate(keys)})
        solver.adjoint(p, N, I, ck, {k: seeds[i] for i, k in enumerate(keys)}, out=d_out, stride=K or None)
        for k in h_out:
            h_out[k].copy_(d_out[k], non_blocking=True)
        h_loss.copy_(loss, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    step()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    t = (time.perf_counter() - t0) / args.steps
    t = max_over_ranks(ws, t)
    del ck, d_out
    return {"value": ws * 2 * sc.m * I * N / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": round(t * 1e3, 2)}


# ----------------------------------------------------------------------------- keyframe scale

def run_keyframe(args, local):
    """The paper's keyframe example at its scale (Sec. "Keyframe Simulation": 900 steps,
    forces per particle per step on an 8,002-vertex garment): a 90x90 cloth (8,100
    vertices) draped over the sphere for 900 steps x 20 iterations; targets at steps 300,
    600 and 900 come from a run driven by the scene's global and wind forces; the controls
    are a force per vertex per step starting at zero (21.9M values), differentiated with
    sparse checkpoints (every 30 steps)."""
    import torch
    from paper_2301_01396_gb300 import binding
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N, I, K, keys = 900, 20, 30, (300, 600, 900)
    sc = scenes.sphere_cloth(90, steps=N, iters=I)
    solver = binding.Solver.from_scene(sc)
    x0 = torch.as_tensor(sc.x0.astype(np.float32), device=dev)
    v0 = torch.as_tensor(sc.v0.astype(np.float32), device=dev)
    p_true = binding.params_from_scene(sc, device=dev)
    ck = new_checkpoints(solver, N, K, dev)
    run_forward(solver, p_true, N, I, x0, v0, ck, K)
    targets = {ck_index(N, K, k): solver.read_state(ck, ck_index(N, K, k))[0].clone() for k in keys}
    fvs = torch.zeros((N, sc.V, 3), dtype=torch.float32, device=dev)
    params = binding.Params(dt=p_true.dt, compliance=p_true.compliance, gravity=p_true.gravity,
                            collider_flags=p_true.collider_flags, plane_h=p_true.plane_h, sphere=p_true.sphere,
                            contact_compliance=p_true.contact_compliance, thickness=p_true.thickness,
                            f_vertex_steps=fvs)
    want = ("compliance", "x0", "v0", "f_vertex_steps")
    grads = {k: torch.empty(s, dtype=torch.float64, device=dev)
             for k, s in dict(compliance=(sc.m,), x0=(sc.V, 3), v0=(sc.V, 3), f_vertex_steps=(N, sc.V, 3)).items()}
    box = {}

    def fwd():
        run_forward(solver, params, N, I, x0, v0, ck, K)

    def bwd():
        loss, seeds = solver.loss(ck, targets)
        solver.adjoint(params, N, I, ck, {k: seeds[i] for i, k in enumerate(keys)}, out=grads, stride=K)
        box["loss"] = loss

    for _ in range(max(args.warmup, 1)):
        fwd()
        bwd()
    torch.cuda.synchronize()
    solver.sync_status()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_f = t_b = 0.0
    for _ in range(args.steps):
        ev[0].record()
        fwd()
        ev[1].record()
        bwd()
        ev[2].record()
        torch.cuda.synchronize()
        t_f += ev[0].elapsed_time(ev[1])
        t_b += ev[1].elapsed_time(ev[2])
    t_f, t_b = t_f / args.steps / 1e3, t_b / args.steps / 1e3
    gnorm = float(grads["f_vertex_steps"].norm().item())
    return {
        "metric": "keyframe example: simulated steps/s (forward + gradient)", "impl": "ours", "mode": "keyframe-scale",
        "value": round(N / (t_f + t_b), 1), "unit": "simulated steps/s", "higher_is_better": True, "n_gpus": 1,
        "steps": args.steps, "data": "synthetic",
        "config": {"workload": f"sphere_cloth_90x90: {sc.V} vertices, {sc.m} constraints, {N} steps x {I} iterations, "
                               f"keyframe loss at {list(keys)}, controls: force per vertex per step "
                               f"({N * sc.V * 3} values) starting at zero, plus compliance/x0/v0 gradients",
                   "checkpoint_stride": K, "states_stored": int(ck.shape[0]),
                   "launches_per_iteration": solver.exec_info()["launches_per_iteration"]},
        "forward_s_per_step": round(t_f / N, 6), "gradient_s_per_step": round(t_b / N, 6),
        "forward_s": round(t_f, 3), "gradient_s": round(t_b, 3),
        "loss": float(box["loss"].item()), "grad_norm_f_vertex_steps": gnorm,
        "paper_context": "Table (Pants, 8,002 vertices, 32-core CPU, implicit adjoint): sim forward 0.053, diff "
                         "forward 0.192, matrix assembly 0.050, CG solve 0.254 s/step",
    }


# ----------------------------------------------------------------------------- implicit adjoint

def run_implicit(args, local):
    """The paper's implicit adjoint next to the discrete one on the 256^2 ground cloth (one
    diagonal, bending, ground plane; 40 steps x 30 iterations, contacts from step ~20):
    time per simulated step of each, conjugate-gradient iterations, and how far the two
    gradients are apart (they differ by design: XPBD's end state is not the exactly solved
    step the implicit adjoint differentiates)."""
    import torch
    from paper_2301_01396_gb300 import binding
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    N = args.sim_steps or 40
    sc = scenes.ground_cloth(args.implicit_grid, steps=N)
    solver = binding.Solver.from_scene(sc)
    p = binding.params_from_scene(sc, device=dev)
    x0 = torch.as_tensor(sc.x0.astype(np.float32), device=dev)
    v0 = torch.as_tensor(sc.v0.astype(np.float32), device=dev)
    I = sc.iters
    ck = solver.forward(p, N, I, x0, v0)
    rng = np.random.default_rng(3)
    seed = {N: torch.as_tensor(rng.standard_normal((sc.V, 3)).astype(np.float32), device=dev)}
    want = ("compliance", "x0", "v0", "f_global", "f_vertex")
    n = args.implicit_grid
    mg = {"multigrid": (n, n, 1, args.mg_sweeps), "multigrid-points": (n, n, 0, args.mg_sweeps),
          "jacobi": None}[args.implicit_precond]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    solver.adjoint(p, N, I, ck, seed, want=want)   # warm-up (allocations)
    solver.adjoint_implicit(p, N, I, ck, seed, want=want, cg_tol=args.cg_tol, cg_max_iters=20000, multigrid=mg)
    torch.cuda.synchronize()
    ev[0].record()
    solver.forward(p, N, I, x0, v0, checkpoints=ck)
    ev[1].record()
    gd = solver.adjoint(p, N, I, ck, seed, want=want)
    ev[2].record()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gi, its = solver.adjoint_implicit(p, N, I, ck, seed, want=want, cg_tol=args.cg_tol, cg_max_iters=20000,
                                      multigrid=mg)
    ev[3].record()
    torch.cuda.synchronize()
    t_imp = (time.perf_counter() - t0) * 1e3
    solver.sync_status()
    diff = {}
    for k in want:
        a, b = gi[k].double(), gd[k].double()
        diff[k] = float((a - b).norm() / b.norm().clamp_min(1e-300))
    return {
        "metric": "implicit adjoint: ms per simulated step", "impl": "ours", "mode": "implicit",
        "value": round(t_imp / N, 3), "unit": "ms/step", "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
        "config": {"workload": f"ground_cloth_{args.implicit_grid}x{args.implicit_grid}: {sc.V} vertices, {sc.m} "
                               f"constraints, {N} steps x {I} iterations, ground plane",
                   "cg_tol": args.cg_tol, "pd_project": True,
                   "preconditioner": {"jacobi": "block Jacobi (3x3 per vertex)",
                                      "multigrid": f"grid multigrid V-cycle, diagonal-line Gauss-Seidel on the "
                                                   f"finest level, {args.mg_sweeps} sweep(s)",
                                      "multigrid-points": f"grid multigrid V-cycle, point Gauss-Seidel, "
                                                          f"{args.mg_sweeps} sweep(s)"}[args.implicit_precond]},
        "forward_ms_per_step": round(ev[0].elapsed_time(ev[1]) / N, 3),
        "discrete_adjoint_ms_per_step": round(ev[1].elapsed_time(ev[2]) / N, 3),
        "implicit_adjoint_ms_per_step": round(t_imp / N, 3),
        "cg_iterations": {"mean": round(float(np.mean(its)), 1), "max": int(np.max(its)), "min": int(np.min(its)),
                          "per_step": [int(k) for k in its]},
        "relative_difference_implicit_vs_discrete": diff,
    }


# ----------------------------------------------------------------------------- material estimation

def material_scene(kind: str, tile: int = 8, grid: int = 256, steps: int = 100):
    """The material-estimation workloads.  Tets: the 32^3-cell block of 164k tets (35,937
    vertices) falling onto the ground, 120 steps x 20 iterations at dt = 1/120, inverse
    moduli log-uniform in 1e-6..1e-3 (each tet's pair by one 2x2 solve for "tets-coupled").
    Membrane: a 256^2 sheet (65,536 vertices, 130,050 orthotropic StVK triangles and
    129,540 dihedral bending hinges, tiled coloring with tile^2 blocks) falling flat onto the
    ground at y = -0.6, 100 steps x 30 iterations at dt = 1/60 (the cloth
    material-estimation size)."""
    if kind == "membrane":
        sc = scenes.membrane_cloth(grid, pins=(), steps=steps, iters=30, seed=9, coloring="tiled", tile=tile)
        sc.collider_flags = scenes.COLLIDE_PLANE
        sc.plane_h = -0.6
        return sc
    sc = scenes.tet_block(32, steps=120, iters=20)
    return scenes.couple_tets(sc) if kind == "tets-coupled" else sc


def class_roofline(stats: dict, steps: int):
    """Dominant kernel class by CUDA-event time, its roofline (algorithmic bytes per launch
    over the mean launch time) and the per-class byte rates."""
    timed = {k: v for k, v in stats.items() if v["timed_launches"] > 0 and v["alg_bytes"] > 0}
    dom = max(timed, key=lambda k: timed[k]["ms"])
    d = timed[dom]
    avg_ms = d["ms"] / d["timed_launches"]
    upl = d["units"] / d["launches"]
    bpl = d["alg_bytes"] / d["launches"]
    achieved = bpl / (avg_ms / 1e3) / 1e9
    peak, peak_kind = measured_peak()
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "kernel": dom,
                "launch_avg_ms": round(avg_ms, 4), "units_per_launch": round(upl),
                "bytes_per_unit": round(bpl / upl, 2), "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": round(bpl)}
    class_bytes = {k: {"bytes_per_unit": round(v["alg_bytes"] / v["units"], 2),
                       "gbs": round(v["alg_bytes"] * v["timed_launches"] / v["launches"] / (v["ms"] / 1e3) / 1e9, 1)}
                   for k, v in timed.items() if v["units"] > 0}
    breakdown = {k: round(v["ms"] / steps, 2) for k, v in sorted(stats.items(), key=lambda kv: -kv[1]["ms"])
                 if v["ms"] > 0}
    return roofline, class_bytes, breakdown


def run_material(args, local):
    """One bench step = forward with per-step checkpoints, the loss at the last step against
    a target from perturbed parameters, and the reverse sweep with the material gradients:
    dL/d(a, b) of 100 materials for the tets (mu = a^2, lambda = b^2), dL/d(C00, C11, C01,
    C22) per triangle and dL/d(bending compliance) for the membrane.  Constraint updates
    count scalar constraint rows: a tet pair is 2, a membrane triangle 3."""
    import torch
    from paper_2301_01396_gb300 import binding
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = material_scene(args.material, args.material_tile, args.material_grid)
    if args.sim_steps:
        sc.steps = args.sim_steps
    if args.iters:
        sc.iters = args.iters
    N, I = sc.steps, sc.iters
    solver = binding.Solver.from_scene(sc)
    x0 = torch.as_tensor(sc.x0.astype(np.float32), device=dev)
    v0 = torch.as_tensor(sc.v0.astype(np.float32), device=dev)
    p = binding.params_from_scene(sc, device=dev)
    rng = np.random.default_rng(12)
    want = ("compliance", "x0", "v0")
    tets = args.material != "membrane"
    if tets:
        mat, a, b = scenes.tet_materials(sc.n_tet, 100, seed=6)
        d_mat = torch.as_tensor(mat, device=dev)
        d_a, d_b = [torch.as_tensor(np.asarray(t, np.float32), device=dev) for t in (a, b)]
        comp_true = p.compliance.clone()
        solver.material_compliance(d_mat, d_a * 1.1, d_b * 0.9, comp_true)
        p_true = binding.Params(**{**p.__dict__, "compliance": comp_true})
        solver.material_compliance(d_mat, d_a, d_b, p.compliance)
    else:
        want = want + ("memb_stiffness",)
        K_true = p.memb_stiffness * torch.as_tensor(np.exp(0.2 * rng.standard_normal((sc.n_memb, 1))),
                                                    dtype=torch.float32, device=dev)
        p_true = binding.Params(**{**p.__dict__, "memb_stiffness": K_true.contiguous()})
    ck = solver.forward(p_true, N, I, x0, v0)
    target = solver.read_state(ck, N)[0].clone()
    grads = {}

    def step():
        solver.forward(p, N, I, x0, v0, checkpoints=ck)
        loss, seeds = solver.loss(ck, {N: target})
        g = solver.adjoint(p, N, I, ck, {N: seeds[0]}, want=want)
        if tets:
            g["a"], g["b"] = solver.material_gradient(d_mat, d_a, d_b, g["compliance"])
        grads.update(g)
        grads["loss"] = loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    solver.sync_status()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    solver.profile(True)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    stats = solver.profile_read()
    solver.profile(False)
    solver.sync_status()
    ms = e0.elapsed_time(e1) / args.steps
    rows = sc.m + 3 * sc.n_memb
    units = 2 * rows * I * N
    roofline, class_bytes, breakdown = class_roofline(stats, args.steps)
    if tets:
        wl = (f"tet_block_32: {sc.V} vertices, {sc.n_tet} tets ({sc.m} constraints"
              f"{', each pair by one 2x2 solve' if sc.tet_coupled else ''}), {N} steps x {I} iterations, dt=1/120, "
              f"ground plane, 100 materials, gradients for (a, b), compliance, x0, v0")
    else:
        wl = (f"membrane_cloth_{int(round(sc.V ** 0.5))}: {sc.V} vertices, {sc.n_memb} StVK membrane triangles (3 rows each) + "
              f"{sc.n_bend} bending, {N} steps x {I} iterations, dt=1/60, ground plane y=-0.6, gradients for "
              f"(C00, C11, C01, C22) per triangle, bending compliance, x0, v0")
    return {
        "metric": METRIC + " (material estimation)", "impl": "ours", "mode": f"material-{args.material}",
        "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "vs_baseline": None, "dtype": "f32 (f64 gradient reductions)",
        "data": "synthetic",
        "config": {"workload": wl, "V": sc.V, "constraint_rows": rows, "colors": sc.n_colors,
                   "phase_kernels": solver.exec_info()["phases"],
                   **({"profiling_override": f"sim_steps={N} iters={I} (not a bench value)"}
                      if (args.sim_steps or args.iters) else {})},
        "roofline": roofline, "clocks": clk,
        "gpu_launches": int(sum(v["launches"] for v in stats.values())),
        "breakdown_ms_per_step": breakdown, "class_bytes": class_bytes,
        "loss": float(grads["loss"].item()),
    }


# ----------------------------------------------------------------------------- serving

def run_serving(args):
    """Serving stream: seeded cloth requests (side U{32..512}, horizon U{20..200} steps,
    U{10..40} iterations, 0-4 pins on the top row, ground plane with probability 1/2), each
    a forward solve + keyframe loss at the last step + full reverse sweep.  Poisson arrivals
    at `serving-load` x the one-at-a-time service rate (measured on the first requests).
    The same trace is served (a) one request at a time, FIFO, through the one-request API,
    (b) by the continuous-batching server; every request's gradients from (b) are checked
    against (a)."""
    import torch
    from paper_2301_01396_gb300 import binding
    dev = torch.device("cuda")
    trace = scenes.serving_requests(args.serving_requests, seed=5)
    items = []
    for k, rq in enumerate(trace):
        sc = scenes.request_scene(rq)
        solver = binding.Solver.from_scene(sc)
        p = binding.params_from_scene(sc, device=dev)
        rng = np.random.default_rng(1000 + k)
        target = sc.x0 + 0.05 * rng.standard_normal(sc.x0.shape)
        items.append(dict(sc=sc, solver=solver, p=p, x0=torch.as_tensor(sc.x0.astype(np.float32), device=dev),
                          v0=torch.as_tensor(sc.v0.astype(np.float32), device=dev),
                          target=torch.as_tensor(target.astype(np.float32), device=dev)))
    want = ("compliance", "x0", "v0")

    def serve_one(it):
        sc, solver, p = it["sc"], it["solver"], it["p"]
        ck = solver.forward(p, sc.steps, sc.iters, it["x0"], it["v0"])
        loss, seeds = solver.loss(ck, {sc.steps: it["target"]})
        g = solver.adjoint(p, sc.steps, sc.iters, ck, {sc.steps: seeds[0]}, want=want)
        torch.cuda.synchronize()
        return g

    def done_one(it):
        # the next request runs on another handle: give this one's tapes back (thousands of
        # handles each keeping its largest workspace would not fit in device memory)
        it["solver"].release_workspace()

    n_cal = min(6, len(items))
    t0 = time.perf_counter()
    for it in items[:n_cal]:
        serve_one(it)
        done_one(it)
    mean_service = (time.perf_counter() - t0) / n_cal
    rng = np.random.default_rng(55)
    gaps = rng.exponential(mean_service / args.serving_load, len(items))
    arrivals = np.cumsum(gaps) - gaps[0]

    # (a) one request at a time, FIFO, one-request API
    lat_a, ref = [], []
    t0 = time.perf_counter()
    for k, it in enumerate(items):
        now = time.perf_counter() - t0
        if now < arrivals[k]:
            time.sleep(arrivals[k] - now)
        g = serve_one(it)
        lat_a.append(time.perf_counter() - t0 - arrivals[k])
        ref.append({kk: v.cpu() for kk, v in g.items()})
        del g
        done_one(it)
    span_a = time.perf_counter() - t0

    # (b) continuous batching: arrivals are admitted while earlier requests run
    srv = binding.Server(max_slots=args.serving_slots)
    lat_b = [0.0] * len(items)
    tickets = [None] * len(items)
    live = {}
    nxt = 0
    max_active = 0
    t_run = t_poll = 0.0
    t0 = time.perf_counter()
    while nxt < len(items) or live:
        now = time.perf_counter() - t0
        while nxt < len(items) and arrivals[nxt] <= now:
            it = items[nxt]
            sc = it["sc"]
            t = srv.submit(it["solver"], it["p"], sc.steps, sc.iters, it["x0"], it["v0"], it["target"], want=want)
            tickets[nxt] = t
            live[t] = nxt
            nxt += 1
        if not live:
            time.sleep(min(max(arrivals[nxt] - now, 0.0), 0.002))
            continue
        r0 = time.perf_counter()
        max_active = max(max_active, srv.run(args.serving_ticks))
        r1 = time.perf_counter()
        for t in list(live):
            if srv.poll(t):
                k = live.pop(t)
                lat_b[k] = time.perf_counter() - t0 - arrivals[k]
        t_run += r1 - r0
        t_poll += time.perf_counter() - r1
    span_b = time.perf_counter() - t0
    st = srv.stats()
    diffs = []
    for k, t in enumerate(tickets):
        res = srv.result(t)
        dk = 0.0
        for kk in want:
            a, b = res[kk].cpu(), ref[k][kk]
            dk = max(dk, float((a - b).norm() / max(float(b.norm()), 1e-300)))
        diffs.append(dk)
    worst = max(diffs) if diffs else 0.0
    kw = int(np.argmax(diffs)) if diffs else 0
    srv.close()

    def pct(lat):
        return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))

    sim_steps = sum(it["sc"].steps for it in items)
    updates = sum(2 * it["sc"].m * it["sc"].iters * it["sc"].steps for it in items)
    pa, pb = pct(lat_a), pct(lat_b)
    return {
        "metric": "serving p50/p99 latency (s) and simulated steps/s", "impl": "ours", "mode": "serving",
        "n_gpus": 1, "data": "synthetic",
        "config": {"workload": f"serving stream: {len(items)} seeded cloth requests (side 32-512, 20-200 steps, "
                               f"10-40 iterations, forward + loss + full reverse sweep), Poisson arrivals at "
                               f"{args.serving_load} x the one-at-a-time service rate",
                   "requests": len(items), "slots": args.serving_slots, "mean_service_s": round(mean_service, 4)},
        "batched": {"p50_s": round(pb[0], 4), "p99_s": round(pb[1], 4), "makespan_s": round(span_b, 3),
                    "steps_per_s": round(sim_steps / span_b, 1), "updates_per_s": updates / span_b,
                    "max_resident": max_active, "ticks": st["ticks"], "batch_launches": st["batches"],
                    "passes": st["items"], "host_wait_s": round(st["host_wait_s"], 3),
                    "host_build_s": round(st["host_build_s"], 3), "host_run_call_s": round(t_run, 3),
                    "host_poll_s": round(t_poll, 3)},
        "one_at_a_time": {"p50_s": round(pa[0], 4), "p99_s": round(pa[1], 4), "makespan_s": round(span_a, 3),
                          "steps_per_s": round(sim_steps / span_a, 1), "updates_per_s": updates / span_a},
        "speedup_steps_per_s": round(span_a / span_b, 3),
        "max_rel_grad_diff_batched_vs_single": worst,
        "rel_grad_diff_batched_vs_single": {
            "median": float(np.median(diffs)) if diffs else 0.0,
            "p99": float(np.percentile(diffs, 99)) if diffs else 0.0,
            "worst_request": {"side": int(items[kw]["sc"].V ** 0.5 + 0.5), "steps": items[kw]["sc"].steps,
                              "iters": items[kw]["sc"].iters, "ground": bool(items[kw]["sc"].collider_flags)}
            if diffs else None},
    }


# ----------------------------------------------------------------------------- reference arm

def run_reference(args, ws, rank):
    """The FP64 oracle as the reference arm, on the host cores: each step is a bounded
    window sample of the workload (forward + reverse sweep)."""
    if rank != 0:
        return None
    import oracle
    nw, st = args.cpu_window, 1
    for _ in range(args.warmup):
        run_cpu_oracle(nw, st)
    t_units, t_time = 0, 0.0
    for _ in range(args.steps):
        sc = cpu_window_scene(nw, st)
        t0 = time.perf_counter()
        xs, _ = oracle.forward(sc)
        oracle.adjoint(sc, {st: xs[-1] - sc.x0})
        t_time += time.perf_counter() - t0
        t_units += 2 * sc.m * sc.iters * st
    value = t_units / t_time
    sample = (f"{nw}x{nw} window of the {GRID}x{GRID} cloth, 1 step x 15 iterations forward + reverse sweep "
              f"per bench step, FP64")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_time / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"sphere_cloth_{GRID}x{GRID} (bounded window sample)", "window": nw},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores only; other ranks exit without work
        res = run_reference(args, ws, rank)
        if res is not None:
            print(json.dumps(res))
        return
    dist_init(ws)
    if args.serving:
        if rank == 0:
            print(json.dumps(run_serving(args)))
        return
    if args.keyframe_scale:
        if rank == 0:
            print(json.dumps(run_keyframe(args, local)))
        return
    if args.implicit:
        if rank == 0:
            print(json.dumps(run_implicit(args, local)))
        return
    if args.material:
        if rank == 0:
            print(json.dumps(run_material(args, local)))
        return
    res = run_ours(args, ws, rank, local)
    if res is not None and rank == 0:
        print(json.dumps(res))
    if ws > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
